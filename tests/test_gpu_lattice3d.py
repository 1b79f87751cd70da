"""The 3-D lattice colour step that updates every chain of a site in one thread (FP32, 4 or 8
chains; the kernel of the 256^3 workload), against the oracle through the C ABI.

Same seeded inputs and Philox counters as the oracle, so the chains are coupled draw for draw
and compared element by element with |x_gpu - x_oracle| / max(|x_oracle|, 1): <= 1e-5 after one
sweep, <= 1e-4 after longer runs (x, posterior mean, tau and sigma^2 traces).  Extents are
ragged (odd widths, a single plane, a single column), chain counts pad (5 -> 8), and the proper
prior, the intercept, the reduce-only pass of gmrf_hyper_update and CUDA-graph replay are each
exercised.
"""
import numpy as np
import pytest

import oracle
from gmrf_testutil import TOL_FP32_1, TOL_FP32_1000, relerr, run_oracle, trace_relerr
from paper_1702_05518_gb300 import gmrf as g
from paper_1702_05518_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

WIDE = {"wide_3d": 1}
GENERAL = {"wide_3d": -1}
NAME = "colour step, 3-D 6-neighbour lattice, all chains of a site per thread"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1702_05518_gb300 import build

    build.build()


def _run(f, C, T, tuning=WIDE, seed=29, **kw):
    with g.Sampler([f], precision=g.FP32, chains=C, seed=seed, tuning=tuning, **kw) as s:
        s.sweep(T)
        res = [s.fetch(0, c, trace=T) for c in range(C)]
        info = s.info()
    return res, info


def _compare(f, res, C, T, tol, seed=29, **okw):
    st, out = run_oracle(f, C, T, seed=seed, stream=0, **okw)
    for c in range(C):
        assert relerr(res[c]["x"], st.x[c]) <= tol, c
        assert trace_relerr(res[c]["tau_trace"], out["tau_trace"][c]) <= tol, c
        assert trace_relerr(res[c]["sigma2_trace"], out["sigma2_trace"][c]) <= tol, c
    return st, out


CASES = [
    ("17x12x33_c8", (17, 12, 33), 8, {}),
    ("9x10x11_c4", (9, 10, 11), 4, {}),
    ("5x7x130_c5", (5, 7, 130), 5, {}),
    ("1x1x9_c8", (1, 1, 9), 8, {}),
    ("4x6x1_c8", (4, 6, 1), 8, {}),
    ("1x1x1_c4", (1, 1, 1), 4, {}),
    ("13x9x20_c8_pcar", (13, 9, 20), 8, {"prior": "pcar", "rho": 0.9}),
    ("40x33x65_c8", (40, 33, 65), 8, {}),
]


@pytest.mark.parametrize("name,dims,C,mk", CASES, ids=[c[0] for c in CASES])
def test_one_sweep(name, dims, C, mk):
    f = wl.small_lattice(wl.LATTICE3D_6, dims, 4)
    prior = g.PRIOR_PCAR if mk.get("prior") == "pcar" else g.PRIOR_ICAR
    res, _ = _run(f, C, 1, prior=prior, rho=mk.get("rho", 1.0))
    _compare(f, res, C, 1, TOL_FP32_1, **mk)


@pytest.mark.parametrize("C", [4, 8])
def test_accumulated_run(C):
    f = wl.small_lattice(wl.LATTICE3D_6, (21, 14, 37), 6)
    res, info = _run(f, C, 60, burn_in=20, graph_sweeps=7)
    st, _ = _compare(f, res, C, 60, TOL_FP32_1000, burn_in=20)
    for c in range(C):
        assert relerr(res[c]["mean"], st.mean[c]) <= TOL_FP32_1000
        assert relerr(res[c]["var"], st.m2[c] / (st.count - 1)) <= 1e-3
    assert info["accumulated"] == 40


def test_intercept():
    f = wl.small_lattice(wl.LATTICE3D_6, (15, 16, 17), 7)
    f = dict(f, y=f["y"] + 3.0)
    with g.Sampler([f], precision=g.FP32, chains=8, seed=31, tuning=WIDE, intercept=True) as s:
        s.sweep(30)
        res = [s.fetch(0, c, trace=30) for c in range(8)]
        b = [s.fetch_intercept(0, c, trace=30) for c in range(8)]
    st, out = run_oracle(f, 8, 30, seed=31, stream=0, intercept=True)
    for c in range(8):
        assert relerr(res[c]["x"], st.x[c]) <= TOL_FP32_1000
        assert trace_relerr(res[c]["tau_trace"], out["tau_trace"][c]) <= TOL_FP32_1000
        assert relerr(b[c]["beta0_trace"], out["beta0_trace"][c]) <= TOL_FP32_1000


def test_reduce_only_hyper_draw():
    f = wl.small_lattice(wl.LATTICE3D_6, (10, 11, 12), 8)
    C = 8
    x0 = wl.rng(2).normal(0, 1, (C, f["n"]))
    f = dict(f, x0=x0)
    with g.Sampler([f], precision=g.FP32, chains=C, seed=37, tuning=WIDE, a_tau=2.0, b_tau=0.5,
                   a_sigma=3.0, b_sigma=0.25) as s:
        s.hyper_update()
        got = [s.fetch(0, c) for c in range(C)]
    rp, ci = oracle.lattice_csr(oracle.LAT3D_6, f["dims"])
    rank = f["n"] - oracle.components(rp, ci)
    for c in range(C):
        x32 = x0[c].astype(np.float32).astype(np.float64)
        S = oracle.quadform(rp, ci, x32)
        R = float(np.sum((f["y"].astype(np.float32).astype(np.float64) - x32) ** 2))
        tau, _ = oracle.gamma_draw(2.0 + rank / 2, 0.5 + S / 2, 37, 0, 0, 5, c)
        prec, _ = oracle.gamma_draw(3.0 + f["n"] / 2, 0.25 + R / 2, 37, 0, 0, 6, c)
        assert got[c]["tau"] == pytest.approx(tau, rel=1e-5)
        assert got[c]["sigma2"] == pytest.approx(1 / prec, rel=1e-5)
        assert np.array_equal(got[c]["x"], x32)


def test_graph_replay_equals_direct_launches():
    f = wl.small_lattice(wl.LATTICE3D_6, (18, 19, 20), 9)
    a, _ = _run(f, 8, 12, graph_sweeps=5)
    b, _ = _run(f, 8, 12, graph_sweeps=0)
    for c in range(8):
        assert np.array_equal(a[c]["x"], b[c]["x"])
        assert np.array_equal(a[c]["tau_trace"], b[c]["tau_trace"])


def test_general_kernel_agrees_and_selection():
    f = wl.small_lattice(wl.LATTICE3D_6, (12, 40, 41), 10)
    a, _ = _run(f, 8, 10, tuning=WIDE)
    b, _ = _run(f, 8, 10, tuning=GENERAL)
    for c in range(8):
        assert relerr(a[c]["x"], b[c]["x"]) <= 2 * TOL_FP32_1000
    with g.Sampler([f], precision=g.FP32, chains=8, seed=1, tuning=WIDE, graph_sweeps=0) as s:
        names = [s.launch_stage(k) for k in range(s.info()["launches_per_sweep"])]
    assert names.count(NAME) == 2
    with g.Sampler([f], precision=g.FP32, chains=8, seed=1, graph_sweeps=0) as s:  # small: general kernel
        names = [s.launch_stage(k) for k in range(s.info()["launches_per_sweep"])]
    assert NAME not in names


@pytest.mark.parametrize("bad", [{"wide_3d": 2}, {"wide_3d": -2}])
def test_invalid_wide_tuning(bad):
    f = wl.small_lattice(wl.LATTICE3D_6, (4, 4, 4), 1)
    with pytest.raises(g.GmrfError):
        g.Sampler([f], precision=g.FP32, chains=8, seed=1, tuning=bad)
    with pytest.raises(g.GmrfError):  # one chain or FP64: not available
        g.Sampler([f], precision=g.FP32, chains=2, seed=1, tuning=WIDE)
    with pytest.raises(g.GmrfError):
        g.Sampler([f], precision=g.FP64, chains=8, seed=1, tuning=WIDE)


def test_normals_timing_diagnostic():
    # the random numbers of a 256^3 colour step with 8 chains alone: a few tens of microseconds,
    # and about half that for 4 chains (one Philox block per site instead of two)
    t8 = g.normals_timing(5, 1 << 23, 8, reps=5)
    t4 = g.normals_timing(5, 1 << 23, 4, reps=5)
    assert 5.0 < t8 < 5000.0 and 0.3 * t8 < t4 < 0.9 * t8
    with pytest.raises(g.GmrfError):
        g.normals_timing(5, 0, 8)
    with pytest.raises(g.GmrfError):
        g.normals_timing(5, 100, 9)
