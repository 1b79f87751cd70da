"""GPU chain diagnostics against the oracle's statements of them, on the GPU's own traces.

The IAT (Geyer's initial monotone sequence), ESS and PSRF computed on the device from the
tau^2, sigma^2, tau and beta0 traces must equal the oracle's on the same values (FP64: to
rounding, 1e-9 relative); the per-site PSRF from the running moments must equal the oracle's
formula on the fetched per-chain means and variances.
"""
import numpy as np
import pytest

import oracle
from paper_1702_05518_gb300 import gmrf as g
from paper_1702_05518_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1702_05518_gb300 import build

    build.build()


def _field():
    f = wl.small_lattice(wl.LATTICE2D_8, (23, 29), 11)
    return dict(f, y=f["y"] + 2.0)


@pytest.mark.parametrize("precision", [g.FP64, g.FP32])
def test_trace_diagnostics_match_oracle(precision):
    C, T = 4, 400
    f = _field()
    with g.Sampler([f], precision=precision, chains=C, seed=91, trace_capacity=300, intercept=True,
                   graph_sweeps=20) as s:
        s.sweep(T)
        fetched = [dict(s.fetch(0, c, trace=300), **s.fetch_intercept(0, c, trace=300)) for c in range(C)]
        for param, key, fn in [(g.PARAM_TAU2, "tau_trace", lambda v: 1.0 / v), (g.PARAM_TAU, "tau_trace", None),
                               (g.PARAM_SIGMA2, "sigma2_trace", None), (g.PARAM_BETA0, "beta0_trace", None)]:
            for n_last in (0, 150, 10_000):
                d = s.trace_diagnostics(0, param, n_last)
                N = 300 if n_last in (0, 10_000) else n_last
                tr = np.stack([fetched[c][key][-N:] for c in range(C)])
                if fn:
                    tr = fn(tr)
                for c in range(C):
                    want = oracle.iat(tr[c])
                    assert d["iat"][c] == pytest.approx(want, rel=1e-9), (param, n_last, c)
                    assert d["ess"][c] == pytest.approx(N / want, rel=1e-9)
                assert d["psrf"] == pytest.approx(oracle.psrf(tr), rel=1e-9)


def test_site_psrf_matches_oracle():
    C = 3
    f = _field()
    with g.Sampler([f], precision=g.FP64, chains=C, seed=93, burn_in=50, graph_sweeps=10) as s:
        s.sweep(200)
        got, mx = s.site_psrf(0)
        parts = [s.fetch(0, c) for c in range(C)]
        k = s.info()["accumulated"]
    means = np.stack([p["mean"] for p in parts])
    vars_ = np.stack([p["var"] for p in parts])
    want = np.array([oracle.psrf_moments(means[:, i], vars_[:, i], k) for i in range(f["n"])])
    np.testing.assert_allclose(got, want, rtol=1e-12)
    assert mx == pytest.approx(np.nanmax(want), rel=1e-15)
    assert np.all(want > 0.5) and k == 150


def test_site_psrf_csr_fp32():
    rp, ci, _ = wl.delaunay_graph(1200, wl.rng(8))
    f = wl.graph_field(rp, ci, seed=108)
    f["color_seed"] = 8
    with g.Sampler([f], precision=g.FP32, chains=2, seed=95, burn_in=20) as s:
        s.sweep(120)
        got, mx = s.site_psrf(0)
        parts = [s.fetch(0, c) for c in range(2)]
        k = s.info()["accumulated"]
    means = np.stack([p["mean"] for p in parts])
    vars_ = np.stack([p["var"] for p in parts])
    want = np.array([oracle.psrf_moments(means[:, i], vars_[:, i], k) for i in range(f["n"])])
    np.testing.assert_allclose(got, want, rtol=1e-12)


def test_diagnostics_errors():
    f = _field()
    with g.Sampler([f], precision=g.FP64, chains=1, seed=1) as s:
        s.sweep(10)
        with pytest.raises(g.GmrfError):
            s.site_psrf(0)  # one chain
        with pytest.raises(g.GmrfError):
            s.trace_diagnostics(0, g.PARAM_BETA0)  # no intercept
        d = s.trace_diagnostics(0, g.PARAM_TAU2)
        assert np.isnan(d["psrf"]) and np.isfinite(d["iat"][0])
    with g.Sampler([f], precision=g.FP64, chains=2, seed=1, burn_in=100) as s:
        s.sweep(10)
        with pytest.raises(g.GmrfError):
            s.site_psrf(0)  # nothing accumulated yet
        with pytest.raises(g.GmrfError):
            s.trace_diagnostics(0, 7)
