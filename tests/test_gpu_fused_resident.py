"""The resident form of the fused 2-D lattice sweep (FP32 samplers of one field whose tiles fit in
one wave, every thread holding all chains): whole batches of sweeps in one cooperative launch, a
grid barrier per sweep, every block drawing tau, sigma^2 (and beta0) of every chain from all tile
partials in the order of the draw kernel.

It runs the per-sweep path's arithmetic in the same order, so its results must equal that path's
(GMRF_FLAG_NO_RESIDENT) bit for bit: states of every chain, running means and variances, the
tau, sigma^2 and beta0 traces, across batch boundaries and split calls, for both lattice kinds,
1, 2 and 4 chains per thread, the proper prior and the intercept.  Parity with the oracle
(Algorithm 1, Sec. 3.1 conditionals) at the FP32 bars, and a barrier wait that runs out reports
GMRF_E_TIMEOUT.
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


def _run(f, C, calls, flags=0, intercept=False, **kw):
    kw.setdefault("burn_in", 40)
    with g.Sampler([f], precision=g.FP32, chains=C, seed=311, flags=flags, intercept=intercept, **kw) as s:
        info = s.info()
        for n in calls:
            s.sweep(n)
        total = sum(calls)
        out = []
        for c in range(C):
            r = s.fetch(0, c, trace=total)
            if intercept:
                r.update(s.fetch_intercept(0, c, trace=total))
            out.append(r)
        after = s.info()
    return out, info, after


def _same(a, b, intercept=False):
    for ra, rb in zip(a, b):
        for k in ("x", "mean", "var", "tau_trace", "sigma2_trace"):
            assert np.array_equal(ra[k], rb[k]), k
        assert ra["tau"] == rb["tau"] and ra["sigma2"] == rb["sigma2"]
        if intercept:
            assert np.array_equal(ra["beta0_trace"], rb["beta0_trace"]) and ra["beta0"] == rb["beta0"]


CASES = [  # (kind, dims, chains, extra sampler arguments)
    (wl.LATTICE2D_8, (512, 512), 3, dict(intercept=True)),  # the paper's p = 512 image model
    (wl.LATTICE2D_8, (300, 244), 2, dict(prior=g.PRIOR_PCAR, rho=0.9)),
    (wl.LATTICE2D_4, (1024, 1024), 1, {}),
    (wl.LATTICE2D_4, (257, 131), 2, {}),
    (wl.LATTICE2D_4, (300, 244), 4, dict(intercept=True)),
    (wl.LATTICE2D_8, (130, 1001), 4, {}),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{'8' if k == wl.LATTICE2D_8 else '4'}nbr-{d[0]}x{d[1]}-C{c}"
                                             for k, d, c, _ in CASES])
def test_fused_resident_equals_per_sweep_path(case):
    kind, dims, C, kw = case
    f = wl.small_lattice(kind, dims, 51)
    if kw.get("intercept"):
        f = dict(f, y=f["y"] + 2.0)
    calls = [37, 70, 1, 92]  # batch boundaries, a single sweep and a batch cut short
    a, ia, aa = _run(f, C, calls, **kw)
    b, ib, _ = _run(f, C, calls, flags=g.FLAG_NO_RESIDENT, **kw)
    assert ia["resident"] == 4 and ib["resident"] == 0
    _same(a, b, intercept=kw.get("intercept", False))
    assert aa["wait_timeouts"] == 0 and aa["hyper_fallbacks"] == 0


@pytest.mark.parametrize("graph_sweeps", [0, 200])
def test_fused_resident_graph_and_direct_launches(graph_sweeps):
    f = wl.small_lattice(wl.LATTICE2D_8, (300, 244), 52)
    a, _, _ = _run(f, 2, [250], graph_sweeps=graph_sweeps, thin=2)
    b, _, _ = _run(f, 2, [250], flags=g.FLAG_NO_RESIDENT, graph_sweeps=graph_sweeps, thin=2)
    _same(a, b)


def test_fused_resident_fixed_hyper_extra_draw_and_reset():
    f = wl.small_lattice(wl.LATTICE2D_4, (300, 244), 53)
    out = []
    for flags in (0, g.FLAG_NO_RESIDENT):
        with g.Sampler([f], precision=g.FP32, chains=2, seed=9, flags=flags) as s:
            s.sweep(15, with_hyper=False)
            s.sweep(20)
            s.hyper_update()
            s.sweep(9)
            s.reset()
            s.sweep(3)
            out.append([s.fetch(0, c, trace=3) for c in range(2)])
    _same(out[0], out[1])


def test_fused_resident_one_sweep_oracle():
    f = wl.small_lattice(wl.LATTICE2D_8, (300, 244), 54)
    r, info, _ = _run(f, 3, [1], burn_in=0)
    assert info["resident"] == 4
    st, out = run_oracle(f, 3, 1, seed=311, stream=0)
    for c in range(3):
        assert relerr(r[c]["x"], st.x[c]) <= TOL_FP32_1
        assert trace_relerr(r[c]["tau_trace"], out["tau_trace"][c]) <= TOL_FP32_1
        assert trace_relerr(r[c]["sigma2_trace"], out["sigma2_trace"][c]) <= TOL_FP32_1


def test_fused_resident_300_sweeps_oracle():
    f = wl.small_lattice(wl.LATTICE2D_4, (257, 131), 55)
    r, _, _ = _run(f, 2, [300], burn_in=100, graph_sweeps=25)
    st, out = run_oracle(f, 2, 300, seed=311, stream=0, burn_in=100)
    for c in range(2):
        assert relerr(r[c]["x"], st.x[c]) <= TOL_FP32_1000
        assert relerr(r[c]["mean"], st.mean[c]) <= TOL_FP32_1000
        assert trace_relerr(r[c]["tau_trace"], out["tau_trace"][c]) <= TOL_FP32_1000
        assert trace_relerr(r[c]["sigma2_trace"], out["sigma2_trace"][c]) <= TOL_FP32_1000


def test_fused_resident_taken_with_the_intercept():
    f = wl.small_lattice(wl.LATTICE2D_8, (300, 244), 59)
    for flags, want in ((0, 4), (g.FLAG_RESIDENT, 4), (g.FLAG_NO_RESIDENT, 0)):
        with g.Sampler([f], precision=g.FP32, chains=2, seed=1, intercept=True, flags=flags) as s:
            assert s.info()["resident"] == want


def test_fused_resident_not_for_fp64_or_beyond_one_wave():
    with g.Sampler([wl.small_lattice(wl.LATTICE2D_8, (300, 244), 56)], precision=g.FP64, chains=2, seed=1) as s:
        assert s.info()["resident"] == 0
    with g.Sampler([wl.small_lattice(wl.LATTICE2D_8, (2048, 2048), 57)], precision=g.FP32, chains=3, seed=1) as s:
        assert s.info()["resident"] == 0


def test_fused_resident_barrier_timeout_reports_and_poisons():
    f = wl.small_lattice(wl.LATTICE2D_8, (300, 244), 58)
    with g.Sampler([f], precision=g.FP32, chains=2, seed=3, flags=g.FLAG_TEST_STALL) as s:
        assert s.info()["resident"] == 4
        s.sweep(10)
        with pytest.raises(g.GmrfError) as e:
            s.fetch(0, 0)
        assert e.value.status == g.E_TIMEOUT
        with pytest.raises(g.GmrfError) as e:
            s.sweep(1)
        assert e.value.status == g.E_STATE
    a, info, after = _run(f, 2, [10], burn_in=0)
    b, _, _ = _run(f, 2, [10], flags=g.FLAG_NO_RESIDENT, burn_in=0)
    assert info["resident"] == 4 and after["wait_timeouts"] == 0
    _same(a, b)
