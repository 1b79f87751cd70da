"""GPU parity of the intercept model of Sec. 3.1 (y = beta0 1 + x + noise, flat prior on beta0)
against the oracle, through the C ABI, draw for draw on the same counters.

Per sweep: the colour steps use b = (y - beta0) / sigma^2; then beta0 | x, sigma^2 is drawn
(normal, mean 1'(y - x)/n, variance sigma^2/n), then tau, and sigma^2 given the new beta0.
Bounds as for the model without intercept (FP64 1e-12; FP32 1e-5 after one sweep, 1e-4 after
1000), applied to x and to the tau, sigma^2 and beta0 traces (beta0 relative to max(|beta0|, 1)).
"""
import numpy as np
import pytest

import oracle
from gmrf_testutil import TOL_FP32_1, TOL_FP32_1000, TOL_FP64, relerr, run_oracle, trace_relerr
from paper_1702_05518_gb300 import gmrf as g
from paper_1702_05518_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1702_05518_gb300 import build

    build.build()


def _shift(f, c):
    return dict(f, y=f["y"] + c)


def _delaunay(npts, seed):
    rp, ci, _ = wl.delaunay_graph(npts, wl.rng(seed))
    f = wl.graph_field(rp, ci, seed=seed + 100)
    f["color_seed"] = seed
    return f


FIELDS = {
    "2d8_fused": lambda: _shift(wl.small_lattice(wl.LATTICE2D_8, (41, 37), 1), 3.0),
    "2d4_fused": lambda: _shift(wl.small_lattice(wl.LATTICE2D_4, (33, 50), 2), -2.0),
    "3d6": lambda: _shift(wl.small_lattice(wl.LATTICE3D_6, (9, 10, 11), 3), 1.5),
    "csr": lambda: _shift(_delaunay(1500, 4), 4.0),
}


def _run_gpu(fields, chains, nsweeps, precision, seed, **kw):
    with g.Sampler(fields, precision=precision, chains=chains, seed=seed, intercept=True, **kw) as s:
        s.sweep(nsweeps)
        res = [[dict(s.fetch(f, c, trace=nsweeps), **s.fetch_intercept(f, c, trace=nsweeps))
                for c in range(chains)] for f in range(len(fields))]
    return res


def _check(field, res_f, chains, nsweeps, seed, stream, tol, **okw):
    st, out = run_oracle(field, chains, nsweeps, seed=seed, stream=stream, intercept=True, **okw)
    for c in range(chains):
        r = res_f[c]
        assert relerr(r["x"], st.x[c]) <= tol
        assert trace_relerr(r["tau_trace"], out["tau_trace"][c]) <= tol
        assert trace_relerr(r["sigma2_trace"], out["sigma2_trace"][c]) <= tol
        assert relerr(r["beta0_trace"], out["beta0_trace"][c]) <= tol
        assert relerr([r["beta0"]], [st.beta0[c]]) <= tol
    return st, out


@pytest.mark.parametrize("name", sorted(FIELDS))
@pytest.mark.parametrize("prior,rho", [("icar", 1.0), ("pcar", 0.9)])
def test_intercept_fp64(name, prior, rho):
    f = FIELDS[name]()
    pr = g.PRIOR_PCAR if prior == "pcar" else g.PRIOR_ICAR
    res = _run_gpu([f], 3, 80, g.FP64, 71, prior=pr, rho=rho, graph_sweeps=16)
    st, out = _check(f, res[0], 3, 80, 71, 0, TOL_FP64, prior=prior, rho=rho)
    assert np.ptp(out["beta0_trace"][0]) > 0  # the intercept moves


@pytest.mark.parametrize("name", sorted(FIELDS))
def test_intercept_fp32_one_sweep(name):
    f = FIELDS[name]()
    res = _run_gpu([f], 2, 1, g.FP32, 73)
    _check(f, res[0], 2, 1, 73, 0, TOL_FP32_1)


@pytest.mark.parametrize("name", ["2d8_fused", "csr"])
def test_intercept_fp32_1000_sweeps(name):
    f = FIELDS[name]()
    res = _run_gpu([f], 1, 1000, g.FP32, 75, graph_sweeps=50)
    _check(f, res[0], 1, 1000, 75, 0, TOL_FP32_1000)


def test_paper_image_model_fp64():
    # Sec. 3.1 simulation: 50 x 50 pixels, true image 5 exp(-|v|^2/2)/pi on [-3, 3]^2 plus N(0, 1)
    # noise, 8-neighbour intrinsic prior, flat intercept, InvGam(0.001, 0.001) on tau^2 and
    # sigma^2 (Gamma(0.001, rate 0.001) on the precisions), three chains.
    p = 50
    truth = wl.paper_image(p)
    y = (truth + wl.rng(17).normal(0.0, 1.0, (p, p))).ravel()
    f = {"kind": wl.LATTICE2D_8, "dims": (p, p), "n": p * p, "y": y}
    hp = dict(a_tau=0.001, b_tau=0.001, a_sigma=0.001, b_sigma=0.001)
    res = _run_gpu([f], 3, 400, g.FP64, 81, graph_sweeps=40, **hp)
    _check(f, res[0], 3, 400, 81, 0, TOL_FP64, a_tau=0.001, b_tau=0.001, a_sig=0.001, b_sig=0.001)


def test_intercept_batched_fields_fp64():
    fields = [FIELDS["2d8_fused"](), FIELDS["csr"](), FIELDS["3d6"]()]
    res = _run_gpu(fields, 2, 30, g.FP64, 77)
    for i, f in enumerate(fields):
        _check(f, res[i], 2, 30, 77, i, TOL_FP64)


def test_intercept_fixed_hyper_draws_beta_only():
    f = FIELDS["csr"]()
    res = _run_gpu([f], 2, 25, g.FP64, 79, fix_hyper=True, tau0=2.0, sigma2_0=0.5)
    st, out = _check(f, res[0], 2, 25, 79, 0, TOL_FP64, fix_hyper=True, tau0=2.0, sigma2_0=0.5)
    assert np.all(out["tau_trace"] == 2.0) and np.all(out["sigma2_trace"] == 0.5)


def test_intercept_resume_is_exact():
    f = FIELDS["2d8_fused"]()
    C, T1, T2 = 2, 30, 20
    with g.Sampler([f], precision=g.FP64, chains=C, seed=83, intercept=True) as s:
        s.sweep(T1 + T2)
        want = [dict(s.fetch(0, c), **s.fetch_intercept(0, c)) for c in range(C)]
    with g.Sampler([f], precision=g.FP64, chains=C, seed=83, intercept=True) as s:
        s.sweep(T1)
        mid = [dict(s.fetch(0, c), **s.fetch_intercept(0, c)) for c in range(C)]
    f2 = dict(f, x0=np.stack([m["x"] for m in mid]), tau0=[m["tau"] for m in mid],
              sigma2_0=[m["sigma2"] for m in mid], beta0=[m["beta0"] for m in mid])
    with g.Sampler([f2], precision=g.FP64, chains=C, seed=83, intercept=True, start_sweep=T1) as s:
        s.sweep(T2)
        got = [dict(s.fetch(0, c), **s.fetch_intercept(0, c)) for c in range(C)]
    for c in range(C):
        assert np.array_equal(got[c]["x"], want[c]["x"])
        assert got[c]["beta0"] == want[c]["beta0"] and got[c]["sigma2"] == want[c]["sigma2"]


def test_intercept_extra_draw():
    f = FIELDS["csr"]()
    C = 2
    x0 = wl.rng(2).normal(4.0, 1.0, (C, f["n"]))
    f = dict(f, x0=x0, beta0=[0.25, -0.5], sigma2_0=[0.8, 1.3])
    hp = dict(a_tau=2.0, b_tau=0.5, a_sigma=3.0, b_sigma=0.25)
    with g.Sampler([f], precision=g.FP64, chains=C, seed=61, intercept=True, **hp) as s:
        s.hyper_update()
        got = [dict(s.fetch(0, c), **s.fetch_intercept(0, c)) for c in range(C)]
    n = f["n"]
    rank = n - oracle.components(f["row_ptr"], f["col_idx"])
    for c in range(C):
        zb = oracle.beta_normal(61, 0, 0, c, tag=8)
        b = float(np.mean(f["y"] - x0[c])) + np.sqrt(f["sigma2_0"][c] / n) * zb
        S = oracle.quadform(f["row_ptr"], f["col_idx"], x0[c])
        R = float(np.sum((f["y"] - b - x0[c]) ** 2))
        tau, _ = oracle.gamma_draw(2.0 + rank / 2, 0.5 + S / 2, 61, 0, 0, 5, c)
        prec, _ = oracle.gamma_draw(3.0 + n / 2, 0.25 + R / 2, 61, 0, 0, 6, c)
        assert got[c]["beta0"] == pytest.approx(b, rel=1e-12, abs=1e-12)
        assert got[c]["tau"] == pytest.approx(tau, rel=1e-12)
        assert got[c]["sigma2"] == pytest.approx(1 / prec, rel=1e-12)


def test_intercept_reset_restores_beta0():
    f = FIELDS["2d4_fused"]()
    with g.Sampler([f], precision=g.FP64, chains=1, seed=5, intercept=True, beta0_0=1.25) as s:
        s.sweep(5)
        a = s.fetch_intercept(0, 0)["beta0"]
        s.reset()
        assert s.fetch_intercept(0, 0)["beta0"] == 1.25
        s.sweep(5)
        assert s.fetch_intercept(0, 0)["beta0"] == a


def test_no_intercept_rejects_fetch():
    f = FIELDS["2d4_fused"]()
    with g.Sampler([f], precision=g.FP64, chains=1, seed=5) as s:
        with pytest.raises(g.GmrfError):
            s.fetch_intercept(0, 0)
