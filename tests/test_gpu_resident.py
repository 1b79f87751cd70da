"""The resident path (whole sweeps of a small 2-D lattice field per launch, one block per chain):
which samplers take it, parity with the oracle on ragged shapes (FP64 within 1e-12 over many
sweeps; FP32 within 1e-5 after one sweep and 1e-4 after 1000 coupled sweeps), the intercept
model, and agreement with the per-sweep kernels, also when one sampler mixes the two paths
(extra hyperparameter draws, sweeps without draws, batches cut at odd sweep counts).
"""
import numpy as np
import pytest

from gmrf_testutil import TOL_FP32_1, TOL_FP32_1000, TOL_FP64, relerr, run_oracle, trace_relerr
from paper_1702_05518_gb300 import gmrf as g
from paper_1702_05518_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1702_05518_gb300 import build

    build.build()


# (name, kind, dims): ragged extents, single rows and columns, each number of positions per
# thread, and the largest fields the path takes (8-neighbour: 1152 positions per class;
# 4-neighbour: 2304).
SHAPES = [("2d8_1x1", wl.LATTICE2D_8, (1, 1)), ("2d8_1x7", wl.LATTICE2D_8, (1, 7)),
          ("2d8_9x2", wl.LATTICE2D_8, (9, 2)), ("2d8_33x31", wl.LATTICE2D_8, (33, 31)),
          ("2d8_50x50", wl.LATTICE2D_8, (50, 50)), ("2d8_71x63", wl.LATTICE2D_8, (71, 63)),
          ("2d4_1x2", wl.LATTICE2D_4, (1, 2)), ("2d4_7x3", wl.LATTICE2D_4, (7, 3)),
          ("2d4_31x33", wl.LATTICE2D_4, (31, 33)), ("2d4_45x44", wl.LATTICE2D_4, (45, 44)),
          ("2d4_64x64", wl.LATTICE2D_4, (64, 64)), ("2d4_72x63", wl.LATTICE2D_4, (72, 63))]


def _field(kind, dims, seed, shift=0.0):
    f = wl.small_lattice(kind, dims, seed)
    return dict(f, y=f["y"] + shift)


def _run(fields, chains, T, precision, seed, **kw):
    with g.Sampler(fields, precision=precision, chains=chains, seed=seed, **kw) as s:
        s.sweep(T)
        res = [s.fetch(0, c, trace=T) for c in range(chains)]
        if kw.get("intercept"):
            for c in range(chains):
                res[c].update(s.fetch_intercept(0, c, trace=T))
        info = s.info()
    return res, info


def _check_oracle(f, res, chains, T, seed, tol, **okw):
    st, out = run_oracle(f, chains, T, seed=seed, stream=0, **okw)
    for c in range(chains):
        assert relerr(res[c]["x"], st.x[c]) <= tol
        assert trace_relerr(res[c]["tau_trace"], out["tau_trace"][c]) <= tol
        assert trace_relerr(res[c]["sigma2_trace"], out["sigma2_trace"][c]) <= tol
        if okw.get("burn_in") is not None and T > okw["burn_in"]:
            assert relerr(res[c]["mean"], st.mean[c]) <= tol
        if okw.get("intercept"):
            scale = max(1.0, float(np.max(np.abs(out["beta0_trace"][c]))))
            assert np.max(np.abs(res[c]["beta0_trace"] - out["beta0_trace"][c])) / scale <= tol
    return st


def test_which_samplers_take_it():
    small8 = wl.small_lattice(wl.LATTICE2D_8, (50, 50), 1)
    small4 = wl.small_lattice(wl.LATTICE2D_4, (64, 64), 1)
    big8 = wl.small_lattice(wl.LATTICE2D_8, (72, 66), 1)      # 1188 positions in a class
    big4 = wl.small_lattice(wl.LATTICE2D_4, (73, 64), 1)      # 2336
    vol = wl.small_lattice(wl.LATTICE3D_6, (8, 8, 8), 1)

    def res(fields, **kw):
        with g.Sampler(fields, seed=1, **kw) as s:
            return s.info()["resident"]

    assert res([small8], chains=3) == 1
    assert res([small4]) == 1
    assert res([small8], precision=g.FP64) == 0
    assert res([small8], precision=g.FP64, flags=g.FLAG_RESIDENT) == 1
    assert res([small8], flags=g.FLAG_NO_RESIDENT) == 0
    assert res([small8], flags=g.FLAG_PER_COLOUR) == 0
    assert res([small8], intercept=True) == 1
    # beyond the small-lattice form: the fused sweep's tiles kept resident, and no form for 3-D
    assert res([big8]) == 4 and res([big4]) == 4 and res([vol]) == 0
    assert res([big8], intercept=True) == 4 and res([big8], flags=g.FLAG_NO_RESIDENT) == 0
    assert res([small8, small4]) == 0
    assert res([small8], algorithm=g.ALGO_PLAIN, precision=g.FP64) == 0


@pytest.mark.parametrize("name,kind,dims", SHAPES, ids=[s[0] for s in SHAPES])
@pytest.mark.parametrize("chains", [1, 3])
def test_fp64_parity(name, kind, dims, chains):
    f = _field(kind, dims, 41)
    res, info = _run([f], chains, 40, g.FP64, seed=7, flags=g.FLAG_RESIDENT, burn_in=10, graph_sweeps=16)
    assert info["resident"] == 1 and info["sweeps_done"] == 40 and info["accumulated"] == 30
    _check_oracle(f, res, chains, 40, 7, TOL_FP64, burn_in=10)


@pytest.mark.parametrize("name,kind,dims", SHAPES, ids=[s[0] for s in SHAPES])
def test_fp32_one_sweep(name, kind, dims):
    f = _field(kind, dims, 42)
    res, info = _run([f], 2, 1, g.FP32, seed=9)
    assert info["resident"] == 1
    _check_oracle(f, res, 2, 1, 9, TOL_FP32_1)


@pytest.mark.parametrize("kind,dims,chains", [(wl.LATTICE2D_8, (50, 50), 3), (wl.LATTICE2D_4, (64, 64), 1),
                                              (wl.LATTICE2D_8, (17, 40), 4)])
def test_fp32_1000_sweeps(kind, dims, chains):
    f = _field(kind, dims, 43)
    res, info = _run([f], chains, 1000, g.FP32, seed=11, burn_in=300, graph_sweeps=100)
    assert info["resident"] == 1 and info["hyper_fallbacks"] == 0
    _check_oracle(f, res, chains, 1000, 11, TOL_FP32_1000, burn_in=300)


@pytest.mark.parametrize("precision,T,tol", [(g.FP64, 60, TOL_FP64), (g.FP32, 1000, TOL_FP32_1000)])
def test_intercept(precision, T, tol):
    f = _field(wl.LATTICE2D_8, (50, 50), 44, shift=3.0)
    res, info = _run([f], 3, T, precision, seed=13, intercept=True, flags=g.FLAG_RESIDENT, burn_in=T // 2,
                     graph_sweeps=50, a_tau=0.001, b_tau=0.001, a_sigma=0.001, b_sigma=0.001)
    assert info["resident"] == 1
    _check_oracle(f, res, 3, T, 13, tol, intercept=True, burn_in=T // 2, a_tau=0.001, b_tau=0.001,
                  a_sig=0.001, b_sig=0.001)


def _sequence(s, steps):
    for op, arg in steps:
        if op == "sweep":
            s.sweep(arg)
        elif op == "sweep_nohyper":
            s.sweep(arg, with_hyper=False)
        elif op == "hyper":
            s.hyper_update()
        elif op == "reset":
            s.reset()


STEPS = [("sweep", 37), ("hyper", None), ("sweep", 5), ("sweep_nohyper", 3), ("sweep", 70), ("hyper", None),
         ("sweep", 1)]


@pytest.mark.parametrize("kind,dims", [(wl.LATTICE2D_8, (33, 31)), (wl.LATTICE2D_4, (45, 44))])
@pytest.mark.parametrize("intercept", [False, True])
def test_agrees_with_per_sweep_kernels(kind, dims, intercept):
    """The same call sequence (odd batch cuts, extra draws through the per-sweep kernels, sweeps
    without draws) on the resident path and on the per-sweep path: FP64 results within 1e-12."""
    f = _field(kind, dims, 45, shift=2.0 if intercept else 0.0)
    out = []
    for flags in (g.FLAG_RESIDENT, g.FLAG_NO_RESIDENT):
        with g.Sampler([f], precision=g.FP64, chains=3, seed=17, flags=flags, burn_in=20, thin=3,
                       graph_sweeps=8, intercept=intercept) as s:
            _sequence(s, STEPS)
            info = s.info()
            r = [s.fetch(0, c, trace=200) for c in range(3)]
            if intercept:
                for c in range(3):
                    r[c].update(s.fetch_intercept(0, c, trace=200))
            out.append((r, info))
    (a, ia), (b, ib) = out
    assert ia["resident"] == 1 and ib["resident"] == 0
    assert ia["sweeps_done"] == ib["sweeps_done"] and ia["accumulated"] == ib["accumulated"]
    for c in range(3):
        for key in ("x", "mean", "var", "tau_trace", "sigma2_trace") + (("beta0_trace",) if intercept else ()):
            assert relerr(a[c][key], b[c][key]) <= TOL_FP64, key


def test_fix_hyper_and_reset():
    f = _field(wl.LATTICE2D_8, (20, 26), 46)
    with g.Sampler([f], precision=g.FP64, chains=2, seed=19, flags=g.FLAG_RESIDENT, fix_hyper=True, tau0=2.0,
                   sigma2_0=0.5) as s:
        s.sweep(30)
        r1 = [s.fetch(0, c, trace=30) for c in range(2)]
        s.reset()
        s.sweep(30)
        r2 = [s.fetch(0, c, trace=30) for c in range(2)]
    st, out = run_oracle(f, 2, 30, seed=19, stream=0, fix_hyper=True, tau0=2.0, sigma2_0=0.5)
    for c in range(2):
        assert np.array_equal(r1[c]["x"], r2[c]["x"])
        assert relerr(r1[c]["x"], st.x[c]) <= TOL_FP64
        assert np.all(r1[c]["tau_trace"] == 2.0) and np.all(r1[c]["sigma2_trace"] == 0.5)


# --------------------------------------------------------------------------------------------
# Graphs: one block per chain, neighbour records, the same draws
# --------------------------------------------------------------------------------------------
def _delaunay(npts, seed, shift=0.0):
    rp, ci, _ = wl.delaunay_graph(npts, wl.rng(seed))
    f = wl.graph_field(rp, ci, seed=seed + 100)
    f["color_seed"] = seed
    f["y"] = f["y"] + shift
    return f


def _wheels(nw, spokes, seed):
    """nw wheels (a hub joined to a cycle of `spokes` rim sites): hubs of degree `spokes`."""
    rows = []
    for w in range(nw):
        hub = w * (spokes + 1)
        rim = [hub + 1 + k for k in range(spokes)]
        for k, r in enumerate(rim):
            rows.append((hub, r))
            rows.append((r, rim[(k + 1) % spokes]))
    n = nw * (spokes + 1)
    adj = [set() for _ in range(n)]
    for a_, b_ in rows:
        adj[a_].add(b_)
        adj[b_].add(a_)
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum([len(s) for s in adj])
    ci = np.concatenate([sorted(s) for s in adj]).astype(np.int32)
    f = wl.graph_field(rp, ci, seed=seed)
    f["color_seed"] = seed
    return f


# sizes for clusters of 1, 4 and 8 blocks per chain
GRAPHS = [("delaunay_1500", lambda: _delaunay(1500, 21)), ("delaunay_9000", lambda: _delaunay(9000, 22)),
          ("delaunay_20000", lambda: _delaunay(20000, 28)),
          ("wheels_16", lambda: _wheels(40, 16, 23)), ("wheels_9", lambda: _wheels(30, 9, 24)),
          ("delaunay_12", lambda: _delaunay(12, 25))]


def test_graphs_which_take_it():
    small = _delaunay(2000, 1)
    big = _delaunay(40000, 2)  # positions do not fit 16 bits

    def res(fields, **kw):
        with g.Sampler(fields, seed=1, **kw) as s:
            return s.info()["resident"]

    assert res([small], chains=8) == 2
    assert res([dict(small, weights=np.ones(len(small["col_idx"])))]) == 0
    assert res([big]) == 0
    assert res([small], precision=g.FP64) == 0
    assert res([small], precision=g.FP64, flags=g.FLAG_RESIDENT) == 2
    assert res([small], flags=g.FLAG_NO_RESIDENT) == 0
    assert res([small, small]) == 0


@pytest.mark.parametrize("name,make", GRAPHS, ids=[g_[0] for g_ in GRAPHS])
@pytest.mark.parametrize("chains", [1, 3])
def test_graph_fp64_parity(name, make, chains):
    f = make()
    res, info = _run([f], chains, 40, g.FP64, seed=7, flags=g.FLAG_RESIDENT, burn_in=10, graph_sweeps=16,
                     prior=g.PRIOR_PCAR, rho=0.95)
    assert info["resident"] == 2 and info["sweeps_done"] == 40 and info["accumulated"] == 30
    assert info["wait_timeouts"] == 0
    _check_oracle(f, res, chains, 40, 7, TOL_FP64, burn_in=10, prior="pcar", rho=0.95)


@pytest.mark.parametrize("name,make", GRAPHS, ids=[g_[0] for g_ in GRAPHS])
def test_graph_fp32(name, make):
    f = make()
    res, info = _run([f], 4, 1, g.FP32, seed=9)
    assert info["resident"] == 2
    _check_oracle(f, res, 4, 1, 9, TOL_FP32_1)


def test_graph_fp32_1000_sweeps_and_intercept():
    f = _delaunay(4000, 26, shift=2.0)
    res, info = _run([f], 2, 1000, g.FP32, seed=11, burn_in=300, graph_sweeps=100, intercept=True)
    assert info["resident"] == 2 and info["hyper_fallbacks"] == 0 and info["wait_timeouts"] == 0
    _check_oracle(f, res, 2, 1000, 11, TOL_FP32_1000, burn_in=300, intercept=True)


@pytest.mark.parametrize("intercept", [False, True])
def test_graph_agrees_with_per_sweep_kernels(intercept):
    f = _delaunay(3000, 27, shift=2.0 if intercept else 0.0)
    out = []
    for flags in (g.FLAG_RESIDENT, g.FLAG_NO_RESIDENT):
        with g.Sampler([f], precision=g.FP64, chains=3, seed=17, flags=flags, burn_in=20, thin=3,
                       graph_sweeps=8, intercept=intercept) as s:
            _sequence(s, STEPS)
            info = s.info()
            r = [s.fetch(0, c, trace=200) for c in range(3)]
            if intercept:
                for c in range(3):
                    r[c].update(s.fetch_intercept(0, c, trace=200))
            out.append((r, info))
    (a, ia), (b, ib) = out
    assert ia["resident"] == 2 and ib["resident"] == 0
    assert ia["sweeps_done"] == ib["sweeps_done"] and ia["accumulated"] == ib["accumulated"]
    for c in range(3):
        for key in ("x", "mean", "var", "tau_trace", "sigma2_trace") + (("beta0_trace",) if intercept else ()):
            assert relerr(a[c][key], b[c][key]) <= TOL_FP64, key
