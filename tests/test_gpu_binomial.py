"""GPU parity of the binomial model with the logistic link (Sec. 3.2; Polya-Gamma
augmentation) against the oracle, through the C ABI.

FP64: coupled draw for draw (the Polya-Gamma accept/reject decisions are taken in FP64 on both
sides), x and the tau and beta0 traces within 1e-12.  FP32: one sweep within 1e-5 (later sweeps
can decouple, since the decisions see the single-precision state), and the posterior of a
three-site model against the exact posterior by quadrature.
"""
import numpy as np
import pytest

from gmrf_testutil import TOL_FP32_1, TOL_FP64, oracle_colors, oracle_graph, relerr, trace_relerr
import oracle
from paper_1702_05518_gb300 import gmrf as g
from paper_1702_05518_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1702_05518_gb300 import build

    build.build()


def _field(npts, seed):
    f = wl.binomial_delaunay(seed=seed, npts=npts, trials_range=(1, 24))[0]
    f["color_seed"] = seed
    return f


def _lattice(dims, seed):
    gen = wl.rng(seed)
    n = dims[0] * dims[1]
    m = gen.integers(0, 12, n).astype(np.int32)
    y = gen.binomial(m, 0.35).astype(np.float64)
    return {"kind": wl.LATTICE2D_4, "dims": dims, "n": n, "y": y, "trials": m}


def _run(fields, C, T, precision, seed, **kw):
    with g.Sampler(fields, precision=precision, chains=C, seed=seed, likelihood=g.LIKELIHOOD_BINOMIAL,
                   prior=g.PRIOR_PCAR, rho=0.995, a_tau=1.0, b_tau=1.0, beta0_prior=(0.0, 1000.0), **kw) as s:
        s.sweep(T)
        res = [[dict(s.fetch(f, c, trace=T), **s.fetch_intercept(f, c, trace=T)) for c in range(C)]
               for f in range(len(fields))]
        info = s.info()
    return res, info


def _oracle(f, C, T, seed, stream=0):
    st = oracle.initial_state(f["y"], C, x0=np.zeros(f["n"]))
    out = oracle.run(oracle_graph(f), oracle_colors(f), f["y"], st, seed=seed, nsweeps=T, stream=stream,
                     prior="pcar", rho=0.995, a_tau=1.0, b_tau=1.0, trials=f["trials"], beta0_prior=(0.0, 1000.0),
                     accumulate=False)
    return st, out


@pytest.mark.parametrize("kind", ["csr", "lattice"])
def test_binomial_fp64_coupled(kind):
    f = _field(1500, 3) if kind == "csr" else _lattice((33, 41), 4)
    C, T = 2, 25
    res, info = _run([f], C, T, g.FP64, 17, graph_sweeps=5)
    st, out = _oracle(f, C, T, 17)
    for c in range(C):
        assert relerr(res[0][c]["x"], st.x[c]) <= TOL_FP64
        assert trace_relerr(res[0][c]["tau_trace"], out["tau_trace"][c]) <= TOL_FP64
        assert relerr(res[0][c]["beta0_trace"], out["beta0_trace"][c]) <= TOL_FP64
    assert info["hyper_fallbacks"] == 0 and out["fallbacks"] == 0


def test_binomial_fp32_one_sweep():
    f = _field(2000, 5)
    res, _ = _run([f], 3, 1, g.FP32, 19)
    st, out = _oracle(f, 3, 1, 19)
    for c in range(3):
        assert relerr(res[0][c]["x"], st.x[c]) <= TOL_FP32_1
        assert relerr(res[0][c]["beta0_trace"], out["beta0_trace"][c]) <= TOL_FP32_1


def test_binomial_fp32_posterior_three_sites():
    # the oracle's pin (tests/test_oracle_stats.py) on the GPU: path of three sites, proper CAR
    # rho 0.5, tau fixed at 2, beta0 ~ N(0, 4), trials (6, 0, 9), successes (4, 0, 2)
    rp, ci = wl.path_graph(3)
    f = {"kind": wl.CSR, "dims": (3, 0, 0), "n": 3, "row_ptr": rp, "col_idx": ci,
         "y": np.array([4.0, 0.0, 2.0]), "trials": np.array([6, 0, 9], np.int32), "color_seed": 2}
    from test_oracle_stats import _logistic_posterior_by_quadrature

    mx, mb, _ = _logistic_posterior_by_quadrature(rp, ci, f["trials"], f["y"], 2.0, 0.5, 4.0)
    T = 60_000
    with g.Sampler([f], precision=g.FP32, chains=4, seed=23, likelihood=g.LIKELIHOOD_BINOMIAL,
                   prior=g.PRIOR_PCAR, rho=0.5, fix_hyper=True, tau0=2.0, beta0_prior=(0.0, 4.0),
                   burn_in=2000, graph_sweeps=100, trace_capacity=T) as s:
        s.sweep(T)
        means = np.array([s.fetch(0, c)["mean"] for c in range(4)])
        bt = np.array([s.fetch_intercept(0, c, trace=T)["beta0_trace"][2000:] for c in range(4)])
    # four independent chains: their spread gives the standard error of the pooled mean
    se_x = means.std(0, ddof=1) / 2 + 1e-4
    assert np.all(np.abs(means.mean(0) - mx) < 6 * se_x), (means.mean(0), mx, se_x)
    bm = bt.mean(1)
    assert abs(bm.mean() - mb) < 6 * (bm.std(ddof=1) / 2) + 1e-3


def test_binomial_errors():
    f = _field(300, 6)
    with pytest.raises(g.GmrfError):
        g.Sampler([dict(f, trials=None)], likelihood=g.LIKELIHOOD_BINOMIAL)
    bad = dict(f, y=f["y"].copy())
    bad["y"][0] = bad["trials"][0] + 1
    with pytest.raises(g.GmrfError):
        g.Sampler([bad], likelihood=g.LIKELIHOOD_BINOMIAL)
    with pytest.raises(g.GmrfError):
        g.Sampler([f], likelihood=g.LIKELIHOOD_BINOMIAL, precision=g.FP64, algorithm=g.ALGO_PLAIN)
    with g.Sampler([f], likelihood=g.LIKELIHOOD_BINOMIAL, chains=1) as s:
        s.sweep(2)
        with pytest.raises(g.GmrfError):
            s.hyper_update()
        assert np.isfinite(s.fetch_intercept(0, 0)["beta0"])
