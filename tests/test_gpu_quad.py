"""The quad kernel (single-chain FP32 8-neighbour lattices with a row length that is a multiple
of 4): parity with the oracle on ragged multi-tile shapes, agreement with the general fused
kernel, and the paths that share its tiling (reduce-only passes of the extra draw, intercept).
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


SHAPES = [(300, 244), (257, 128), (9, 16), (1, 4), (2, 8), (130, 1000)]


def _run(f, nsweeps, **kw):
    kw.setdefault("flags", g.FLAG_NO_RESIDENT)  # small shapes would take the resident path
    with g.Sampler([f], precision=g.FP32, chains=1, seed=101, **kw) as s:
        s.sweep(nsweeps)
        r = s.fetch(0, 0, trace=nsweeps)
        names = [s.launch_stage(k) for k in range(s.info()["launches_per_sweep"])]
    return r, names


@pytest.mark.parametrize("dims", SHAPES, ids=[f"{h}x{w}" for h, w in SHAPES])
def test_quad_one_sweep(dims):
    f = wl.small_lattice(wl.LATTICE2D_8, dims, 31)
    r, names = _run(f, 1)
    assert names[0].startswith("fused quad sweep")
    st, out = run_oracle(f, 1, 1, seed=101, stream=0)
    assert relerr(r["x"], st.x[0]) <= TOL_FP32_1
    assert trace_relerr(r["tau_trace"], out["tau_trace"][0]) <= TOL_FP32_1


@pytest.mark.parametrize("dims", [(300, 244), (257, 128)])
def test_quad_300_sweeps(dims):
    f = wl.small_lattice(wl.LATTICE2D_8, dims, 32)
    r, _ = _run(f, 300, graph_sweeps=25, burn_in=100)
    st, out = run_oracle(f, 1, 300, seed=101, stream=0, burn_in=100)
    assert relerr(r["x"], st.x[0]) <= TOL_FP32_1000
    assert relerr(r["mean"], st.mean[0]) <= TOL_FP32_1000
    assert trace_relerr(r["sigma2_trace"], out["sigma2_trace"][0]) <= TOL_FP32_1000


def test_quad_matches_general_fused_kernel():
    f = wl.small_lattice(wl.LATTICE2D_8, (200, 176), 33)
    a, na = _run(f, 50)
    b, nb = _run(f, 50, tuning={"quad_config": -1})
    assert na[0].startswith("fused quad sweep") and nb[0].startswith("fused sweep")
    assert relerr(a["x"], b["x"]) <= TOL_FP32_1000
    assert trace_relerr(a["tau_trace"], b["tau_trace"]) <= TOL_FP32_1000


def test_row_length_not_multiple_of_4_uses_general_kernel():
    f = wl.small_lattice(wl.LATTICE2D_8, (40, 42), 34)
    _, names = _run(f, 2)
    assert names[0].startswith("fused sweep")


def test_quad_extra_draw_and_intercept():
    f = wl.small_lattice(wl.LATTICE2D_8, (150, 124), 35)
    f = dict(f, y=f["y"] + 1.0)
    with g.Sampler([f], precision=g.FP32, chains=1, seed=103, intercept=True, flags=g.FLAG_NO_RESIDENT) as s:
        s.sweep(20)
        s.hyper_update()
        s.sweep(5)
        r = dict(s.fetch(0, 0, trace=25), **s.fetch_intercept(0, 0, trace=25))
    # the oracle has no extra draw: compare the first 20 sweeps' traces and check the rest is finite
    st, out = run_oracle(f, 1, 20, seed=103, stream=0, intercept=True)
    assert trace_relerr(r["tau_trace"][:20], out["tau_trace"][0]) <= TOL_FP32_1000
    assert relerr(r["beta0_trace"][:20], out["beta0_trace"][0]) <= TOL_FP32_1000
    assert np.all(np.isfinite(r["x"])) and np.isfinite(r["beta0"])
