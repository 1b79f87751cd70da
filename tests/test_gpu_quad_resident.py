"""The resident form of the quad kernel (single-chain FP32 8-neighbour lattices whose tiles fit in
one wave): whole batches of sweeps in one cooperative launch, a grid barrier per sweep, every
block drawing tau, sigma^2 (and beta0) from all tile partials in the order of the draw kernel.

It runs the per-sweep path's arithmetic in the same order, so its results must equal that path's
(GMRF_FLAG_NO_RESIDENT) bit for bit: state, running mean and variance, the tau, sigma^2 and beta0
traces, across batch boundaries and split calls.  Parity with the oracle (Algorithm 1, Sec. 3.1
conditionals) at the FP32 bars, and a barrier wait that runs out reports GMRF_E_TIMEOUT.
"""
import numpy as np
import pytest

from gmrf_testutil import TOL_FP32_1, TOL_FP32_1000, relerr, run_oracle, trace_relerr
from paper_1702_05518_gb300 import gmrf as g
from paper_1702_05518_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1702_05518_gb300 import build

    build.build()


def _field(dims, seed, shift=0.0):
    f = wl.small_lattice(wl.LATTICE2D_8, dims, seed)
    return dict(f, y=f["y"] + shift) if shift else f


def _run(f, calls, flags=0, intercept=False, **kw):
    kw.setdefault("burn_in", 40)
    with g.Sampler([f], precision=g.FP32, chains=1, seed=211, flags=flags, intercept=intercept, **kw) as s:
        info = s.info()
        for n in calls:
            s.sweep(n)
        total = sum(calls)
        r = s.fetch(0, 0, trace=total)
        if intercept:
            r.update(s.fetch_intercept(0, 0, trace=total))
        r["info"] = s.info()
    return r, info


def _same(a, b, intercept=False):
    for k in ("x", "mean", "var", "tau_trace", "sigma2_trace"):
        assert np.array_equal(a[k], b[k]), k
    assert a["tau"] == b["tau"] and a["sigma2"] == b["sigma2"]
    if intercept:
        assert np.array_equal(a["beta0_trace"], b["beta0_trace"]) and a["beta0"] == b["beta0"]


SHAPES = [(300, 244), (130, 1000), (257, 128), (1024, 1024)]


@pytest.mark.parametrize("dims", SHAPES, ids=[f"{h}x{w}" for h, w in SHAPES])
def test_resident_equals_per_sweep_path(dims):
    f = _field(dims, 41)
    calls = [37, 70, 1, 92]  # batch boundaries, a single sweep and a batch cut short
    a, ia = _run(f, calls)
    b, ib = _run(f, calls, flags=g.FLAG_NO_RESIDENT)
    assert ia["resident"] == 3 and ib["resident"] == 0
    _same(a, b)
    assert a["info"]["wait_timeouts"] == 0 and a["info"]["hyper_fallbacks"] == 0


@pytest.mark.parametrize("graph_sweeps", [0, 25, 200])
def test_resident_graph_and_direct_launches(graph_sweeps):
    # direct batches (no graphs), graphs of 25 sweeps, and batches of 128 inside graphs of 200
    f = _field((300, 244), 42)
    a, _ = _run(f, [250], graph_sweeps=graph_sweeps)
    b, _ = _run(f, [250], flags=g.FLAG_NO_RESIDENT, graph_sweeps=graph_sweeps)
    _same(a, b)


def test_resident_intercept_and_thinning():
    f = _field((256, 200), 43, shift=2.5)
    kw = dict(intercept=True, burn_in=30, thin=3)
    a, _ = _run(f, [64, 65], **kw)
    b, _ = _run(f, [64, 65], flags=g.FLAG_NO_RESIDENT, **kw)
    _same(a, b, intercept=True)


def test_resident_fixed_hyper_and_sweeps_without_draws():
    f = _field((300, 244), 44)
    for kw in (dict(fix_hyper=True, tau0=3.0, sigma2_0=0.4), {}):
        with g.Sampler([f], precision=g.FP32, chains=1, seed=5, **kw) as s, \
                g.Sampler([f], precision=g.FP32, chains=1, seed=5, flags=g.FLAG_NO_RESIDENT, **kw) as t:
            for smp in (s, t):
                smp.sweep(20, with_hyper=False)
                smp.sweep(30)
            a, b = s.fetch(0, 0, trace=50), t.fetch(0, 0, trace=50)
            _same(a, b)
            assert np.all(a["tau_trace"][:20] == a["tau_trace"][0])


def test_resident_extra_draw_then_sweeps():
    f = _field((300, 244), 45)
    out = []
    for flags in (0, g.FLAG_NO_RESIDENT):
        with g.Sampler([f], precision=g.FP32, chains=1, seed=7, flags=flags) as s:
            s.sweep(20)
            s.hyper_update()
            s.sweep(9)
            s.reset()
            s.sweep(3)
            out.append(s.fetch(0, 0, trace=3))
    _same(out[0], out[1])


def test_resident_one_sweep_oracle():
    f = _field((300, 244), 46)
    r, info = _run(f, [1], burn_in=0)
    assert info["resident"] == 3
    st, out = run_oracle(f, 1, 1, seed=211, stream=0)
    assert relerr(r["x"], st.x[0]) <= TOL_FP32_1
    assert trace_relerr(r["tau_trace"], out["tau_trace"][0]) <= TOL_FP32_1
    assert trace_relerr(r["sigma2_trace"], out["sigma2_trace"][0]) <= TOL_FP32_1


def test_resident_300_sweeps_oracle():
    f = _field((257, 128), 47)
    r, _ = _run(f, [300], burn_in=100, graph_sweeps=25)
    st, out = run_oracle(f, 1, 300, seed=211, stream=0, burn_in=100)
    assert relerr(r["x"], st.x[0]) <= TOL_FP32_1000
    assert relerr(r["mean"], st.mean[0]) <= TOL_FP32_1000
    assert trace_relerr(r["tau_trace"], out["tau_trace"][0]) <= TOL_FP32_1000
    assert trace_relerr(r["sigma2_trace"], out["sigma2_trace"][0]) <= TOL_FP32_1000


def test_resident_not_taken_beyond_one_wave():
    # 2048 x 2048 needs more tiles than blocks that fit at once: the per-sweep quad kernel
    f = _field((2048, 2048), 48)
    with g.Sampler([f], precision=g.FP32, chains=1, seed=1) as s:
        assert s.info()["resident"] == 0
        assert s.launch_stage(0).startswith("fused quad sweep")


def test_resident_barrier_timeout_reports_and_poisons():
    # GMRF_FLAG_TEST_STALL: every barrier expects one arrival more than there are blocks, so the
    # first wait runs out (after 1 ms); the blocks leave their loops and the call reports it
    f = _field((300, 244), 49)
    with g.Sampler([f], precision=g.FP32, chains=1, seed=3, flags=g.FLAG_TEST_STALL) as s:
        assert s.info()["resident"] == 3
        s.sweep(10)
        with pytest.raises(g.GmrfError) as e:
            s.fetch(0, 0)
        assert e.value.status == g.E_TIMEOUT
        with pytest.raises(g.GmrfError) as e:
            s.sweep(1)
        assert e.value.status == g.E_STATE
    # the device is unharmed: the same field without the switch samples as before
    a, info = _run(f, [10], burn_in=0)
    b, _ = _run(f, [10], flags=g.FLAG_NO_RESIDENT, burn_in=0)
    assert info["resident"] == 3 and a["info"]["wait_timeouts"] == 0
    _same(a, b)
