"""Failure handling through the C ABI, made to happen on purpose without faulting the GPU.

- A bounded device wait that runs out: GMRF_FLAG_TEST_STALL makes every colour step of the graph
  cluster kernel expect 16 bytes more than the other blocks send, so each block's wait gives up
  (after 1 ms); the kernel still finishes, the next call that reads the sampler's counters
  returns GMRF_E_TIMEOUT, and the sampler refuses all later work with GMRF_E_STATE.  A sampler
  built afterwards on the same graph runs normally (the device is unharmed).
- Device allocations that fail: gmrf_debug_fail_alloc makes the k-th allocation of a
  gmrf_sampler_create (for every k) or of gmrf_color_graph fail; the call returns GMRF_E_OOM,
  leaves *out NULL and keeps no device memory.
- A poisoned sampler (gmrf_debug_poison, the state after a CUDA error): every later call that
  would touch the device returns GMRF_E_STATE, and destroying it works.
"""
import numpy as np
import pytest

from gmrf_testutil import TOL_FP32_1000, relerr, run_oracle
from paper_1702_05518_gb300 import gmrf as g
from paper_1702_05518_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1702_05518_gb300 import build

    build.build()


def _graph(npts=5000, seed=12):
    rp, ci, _ = wl.delaunay_graph(npts, wl.rng(seed))
    f = wl.graph_field(rp, ci, seed=seed + 100)
    f["color_seed"] = seed
    return f


def _free_bytes():
    import torch

    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_device_wait_timeout_is_reported_and_poisons():
    f = _graph()
    with g.Sampler([f], precision=g.FP32, chains=2, seed=41, flags=g.FLAG_TEST_STALL) as s:
        info = s.info()
        assert info["resident"] == 2  # the graph cluster kernel
        s.sweep(10)
        with pytest.raises(g.GmrfError) as e:
            s.fetch(0, 0)
        assert e.value.status == g.E_TIMEOUT
        for call in (lambda: s.sweep(1), lambda: s.info(), lambda: s.fetch(0, 1), lambda: s.hyper_update()):
            with pytest.raises(g.GmrfError) as e2:
                call()
            assert e2.value.status == g.E_STATE
    # the device is unharmed: the same graph without the switch samples as the oracle does
    with g.Sampler([f], precision=g.FP32, chains=2, seed=41) as s:
        s.sweep(10)
        res = [s.fetch(0, c) for c in range(2)]
        assert s.info()["wait_timeouts"] == 0
    st, _ = run_oracle(f, 2, 10, seed=41, stream=0)
    for c in range(2):
        assert relerr(res[c]["x"], st.x[c]) <= TOL_FP32_1000


def test_every_allocation_failure_of_create_is_reported_without_leak():
    f = wl.small_lattice(wl.LATTICE3D_6, (40, 41, 42), 3)
    kw = dict(precision=g.FP32, chains=4, seed=5, graph_sweeps=4)
    with g.Sampler([f], **kw) as s:  # warm-up: modules loaded, pools settled
        s.sweep(4)
    base = _free_bytes()
    failures = 0
    for k in range(1, 400):
        g.debug_fail_alloc(k)
        try:
            s = g.Sampler([f], **kw)
        except g.GmrfError as e:
            assert e.status == g.E_OOM, str(e)
            failures += 1
            continue
        finally:
            g.debug_fail_alloc(0)
        s.close()  # k is past the last allocation: creation succeeded
        break
    else:
        pytest.fail("creation never succeeded")
    assert failures >= 10  # every allocation point was made to fail once
    assert _free_bytes() >= base - (2 << 20)
    with g.Sampler([f], **kw) as s:
        s.sweep(2)
        assert np.isfinite(s.fetch(0, 0)["x"]).all()


def test_allocation_failure_of_color_graph():
    f = _graph(3000, 13)
    g.debug_fail_alloc(1)
    try:
        with pytest.raises(g.GmrfError) as e:
            g.color_graph(f["row_ptr"], f["col_idx"], seed=1)
        assert e.value.status == g.E_OOM
    finally:
        g.debug_fail_alloc(0)
    cols, k = g.color_graph(f["row_ptr"], f["col_idx"], seed=1)
    assert k >= 2 and len(cols) == f["n"]


def test_poisoned_sampler_refuses_every_device_call():
    f = wl.small_lattice(wl.LATTICE2D_8, (40, 50), 2)
    s = g.Sampler([f], precision=g.FP32, chains=2, seed=3, intercept=True, flags=g.FLAG_NO_RESIDENT)
    s.sweep(3)
    s.debug_poison()
    calls = [lambda: s.sweep(1), lambda: s.hyper_update(), lambda: s.fetch(0, 0), lambda: s.fetch_intercept(0, 0),
             lambda: s.info(), lambda: s.reset(), lambda: s.launch_stage(0), lambda: s.trace_diagnostics(0),
             lambda: s.site_psrf(0), lambda: s.set_data(0, f["y"]), lambda: s.fetch_mean(0, 0)]
    for call in calls:
        with pytest.raises(g.GmrfError) as e:
            call()
        assert e.value.status == g.E_STATE
    s.close()
