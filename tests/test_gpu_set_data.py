"""gmrf_sampler_set_data: a sampler that is given new data restarts exactly as a sampler created
with that data (bit for bit on every chromatic path: quad, fused lattices, colour steps,
intercept, binomial; within 1e-12 on the plain sweep, whose atomic sums vary in order), keeps
the other fields' data, rejects bad data without changing anything, and matches the oracle on
the new data.
"""
import numpy as np
import pytest

from gmrf_testutil import TOL_FP32_1000, TOL_FP64, relerr, run_oracle, trace_relerr
from paper_1702_05518_gb300 import gmrf as g
from paper_1702_05518_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1702_05518_gb300 import build

    build.build()


def _delaunay(npts, seed):
    rp, ci, _ = wl.delaunay_graph(npts, wl.rng(seed))
    f = wl.graph_field(rp, ci, seed=seed + 100)
    f["color_seed"] = seed
    return f


def _binomial(npts, seed):
    f = wl.binomial_delaunay(seed=seed, npts=npts, trials_range=(1, 24))[0]
    f["color_seed"] = seed
    return f


def _new_data(f, seed, binomial=False):
    gen = np.random.default_rng(seed)
    n = f["n"]
    if binomial:
        m = gen.integers(0, 20, n).astype(np.int32)
        return {"y": gen.binomial(m, 0.6).astype(np.float64), "trials": m}
    return {"y": f["y"][::-1].copy() + gen.normal(0.0, 0.5, n)}


BINOM = dict(likelihood=g.LIKELIHOOD_BINOMIAL, prior=g.PRIOR_PCAR, rho=0.995, a_tau=1.0, b_tau=1.0)

CASES = {
    "quad_fp32": (lambda: [wl.small_lattice(wl.LATTICE2D_8, (130, 1000), 5)], dict(precision=g.FP32, chains=1)),
    "2d4_fp64_c2": (lambda: [wl.small_lattice(wl.LATTICE2D_4, (33, 50), 6)], dict(precision=g.FP64, chains=2)),
    "3d6_fp32_c3": (lambda: [wl.small_lattice(wl.LATTICE3D_6, (9, 10, 11), 7)], dict(precision=g.FP32, chains=3)),
    "csr_fp64_intercept": (lambda: [_delaunay(1500, 8)], dict(precision=g.FP64, chains=2, intercept=True)),
    "binomial_fp32": (lambda: [_binomial(1200, 9)], dict(precision=g.FP32, chains=2, **BINOM)),
    "binomial_fp64": (lambda: [_binomial(900, 10)], dict(precision=g.FP64, chains=1, **BINOM)),
    "plain_fp64": (lambda: [_delaunay(800, 11)], dict(precision=g.FP64, chains=2, algorithm=g.ALGO_PLAIN)),
    # the resident paths (small single lattice, small single graph in clusters of 4 blocks)
    "resident_lattice_fp32": (lambda: [wl.small_lattice(wl.LATTICE2D_8, (50, 50), 12)],
                              dict(precision=g.FP32, chains=3, intercept=True)),
    "resident_graph_fp32": (lambda: [_delaunay(9000, 13)], dict(precision=g.FP32, chains=2)),
}


def _result(s, nfields, chains, T):
    out = []
    for fi in range(nfields):
        for c in range(chains):
            r = s.fetch(fi, c, trace=T)
            out.append((r["x"], r["mean"], r["tau_trace"], r["sigma2_trace"]))
    return out


def _same(a, b, tol=0.0):
    for ra, rb in zip(a, b):
        for u, v in zip(ra, rb):
            if tol == 0.0:
                np.testing.assert_array_equal(u, v)
            else:
                assert relerr(u, v) <= tol or (np.isnan(u).all() and np.isnan(v).all())


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("with_x0", [False, True])
def test_set_data_equals_fresh_sampler(case, with_x0):
    make, kw = CASES[case]
    fields = make()
    binomial = kw.get("likelihood") == g.LIKELIHOOD_BINOMIAL
    new = _new_data(fields[0], 77, binomial)
    C = kw["chains"]
    x0 = np.random.default_rng(3).normal(0.0, 1.0, (C, fields[0]["n"])) if with_x0 else None
    T = 6
    seed = 2024
    with g.Sampler(fields, seed=seed, **kw) as a:
        a.sweep(4)
        a.set_data(0, new["y"], new.get("trials"), x0)
        a.sweep(T)
        got = _result(a, len(fields), C, T)
        tr_a = [a.fetch_intercept(0, c, trace=T)["beta0_trace"] for c in range(C)] if (
            kw.get("intercept") or binomial) else None
    fresh = [dict(fields[0], **new)]
    if with_x0:
        fresh[0]["x0"] = x0
    with g.Sampler(fresh, seed=seed, **kw) as b:
        b.sweep(T)
        want = _result(b, len(fields), C, T)
        tr_b = [b.fetch_intercept(0, c, trace=T)["beta0_trace"] for c in range(C)] if tr_a is not None else None
    # the plain sweep sums its reductions with atomics (order varies from run to run): FP64 bound
    _same(got, want, TOL_FP64 if kw.get("algorithm") == g.ALGO_PLAIN else 0.0)
    if tr_a is not None:
        for u, v in zip(tr_a, tr_b):
            np.testing.assert_array_equal(u, v)


def test_set_data_keeps_other_fields():
    """Two fields; new data for field 1 only: both restart, field 0 on its old data."""
    f0 = wl.small_lattice(wl.LATTICE2D_8, (40, 64), 12)
    f1 = _delaunay(700, 13)
    new = _new_data(f1, 5)
    T = 5
    with g.Sampler([f0, f1], precision=g.FP32, chains=2, seed=9) as a:
        a.sweep(3)
        a.set_data(1, new["y"])
        a.sweep(T)
        got = _result(a, 2, 2, T)
    with g.Sampler([f0, dict(f1, **new)], precision=g.FP32, chains=2, seed=9) as b:
        b.sweep(T)
        want = _result(b, 2, 2, T)
    _same(got, want)


def test_set_data_matches_oracle():
    """New data, then sweeps: FP64 parity with the oracle run on that data from the start."""
    f = _delaunay(1000, 14)
    new = _new_data(f, 15)
    T = 20
    with g.Sampler([f], precision=g.FP64, chains=2, seed=31) as s:
        s.sweep(7)
        s.set_data(0, new["y"])
        s.sweep(T)
        res = [s.fetch(0, c, trace=T) for c in range(2)]
    st, out = run_oracle(dict(f, **new), 2, T, seed=31, stream=0)
    for c in range(2):
        assert relerr(res[c]["x"], st.x[c]) <= TOL_FP64
        assert trace_relerr(res[c]["tau_trace"], out["tau_trace"][c]) <= TOL_FP64


def test_set_data_rejects_bad_data():
    f = _delaunay(500, 16)
    with g.Sampler([f], precision=g.FP32, chains=1, seed=4) as s:
        s.sweep(3)
        before = s.fetch_x(0, 0)
        # checked on the device after the upload: any position, the last one included
        for i, v in ((17, np.nan), (f["n"] - 1, np.inf), (0, -np.inf)):
            bad = f["y"].copy()
            bad[i] = v
            with pytest.raises(g.GmrfError, match="y must be finite") as e:
                s.set_data(0, bad)
            assert e.value.status == g.E_INVALID
        with pytest.raises(g.GmrfError, match="x0 must be finite") as e:
            s.set_data(0, f["y"], x0=np.full(f["n"], np.inf))
        assert e.value.status == g.E_INVALID
        x0 = np.tile(f["y"], (1, 1))
        x0[0, -1] = np.nan
        with pytest.raises(g.GmrfError, match="x0 must be finite"):
            s.set_data(0, f["y"], x0=x0)
        with pytest.raises(g.GmrfError) as e:
            s.set_data(1, f["y"])
        assert e.value.status == g.E_INVALID
        np.testing.assert_array_equal(s.fetch_x(0, 0), before)  # nothing changed
        s.sweep(2)
        assert np.all(np.isfinite(s.fetch_x(0, 0)))
    fb = _binomial(400, 17)
    with g.Sampler([fb], precision=g.FP32, chains=1, seed=4, **BINOM) as s:
        with pytest.raises(g.GmrfError) as e:
            s.set_data(0, fb["y"])  # binomial data need trials
        assert e.value.status == g.E_INVALID
        m = fb["trials"].copy()
        y = fb["y"].copy()
        y[np.argmax(m)] = m.max() + 1
        with pytest.raises(g.GmrfError, match=r"successes y must be in \[0, trials\]") as e:
            s.set_data(0, y, m)
        assert e.value.status == g.E_INVALID
        for bad_m in (-1, 4096):
            m2 = m.copy()
            m2[-1] = bad_m
            with pytest.raises(g.GmrfError, match="trials must be in 0..4095"):
                s.set_data(0, np.minimum(fb["y"], np.maximum(m2, 0)), m2)
        s.sweep(2)


def test_fetch_mean_into_pinned_buffer():
    import torch

    f = _delaunay(600, 18)
    with g.Sampler([f], precision=g.FP32, chains=2, seed=3, burn_in=2) as s:
        s.sweep(10)
        buf = torch.empty(f["n"], dtype=torch.float64, pin_memory=True)
        m = s.fetch_mean(0, 1, out=buf.numpy())
        np.testing.assert_array_equal(buf.numpy(), s.fetch(0, 1)["mean"])
        assert m is not None


def test_set_data_on_every_field_restarts_once():
    """set_data on each field of a sampler in turn, then the state: before any sweep it is the
    restart state (x = the new y, no sweep done, empty moments); after sweeps it equals a sampler
    created with all the new data."""
    fields = [wl.small_lattice(wl.LATTICE2D_4, (48, 40), 19), _delaunay(800, 20),
              wl.small_lattice(wl.LATTICE3D_6, (6, 7, 8), 21)]
    news = [_new_data(f, 30 + i) for i, f in enumerate(fields)]
    T = 4
    with g.Sampler(fields, precision=g.FP32, chains=2, seed=12, burn_in=0) as a:
        a.sweep(5)
        for fi, nd in enumerate(news):
            a.set_data(fi, nd["y"])
        assert a.info()["sweeps_done"] == 0 and a.info()["accumulated"] == 0
        for fi, nd in enumerate(news):
            np.testing.assert_array_equal(a.fetch_x(fi, 1), nd["y"].astype(np.float32).astype(np.float64))
        a.sweep(T)
        got = _result(a, 3, 2, T)
    with g.Sampler([dict(f, **nd) for f, nd in zip(fields, news)], precision=g.FP32, chains=2, seed=12,
                   burn_in=0) as b:
        b.sweep(T)
        want = _result(b, 3, 2, T)
    _same(got, want)


# --------------------------------------------------------------------------------------------
# Moments pooled over the chains (gmrf_fetch_pooled)
# --------------------------------------------------------------------------------------------
def _pooled(means, m2s, k):
    means, m2s = np.asarray(means), np.asarray(m2s)
    mu = means.mean(axis=0)
    var = (m2s + k * (means - mu) ** 2).sum(axis=0) / (means.shape[0] * k - 1)
    return mu, var


@pytest.mark.parametrize("kind", ["3d_c5", "2d8_c3", "csr_c4"])
def test_fetch_pooled_equals_chains_combined(kind):
    if kind == "3d_c5":
        f, C = wl.small_lattice(wl.LATTICE3D_6, (9, 14, 23), 3), 5
    elif kind == "2d8_c3":
        f, C = wl.small_lattice(wl.LATTICE2D_8, (37, 41), 4), 3
    else:
        rp, ci, _ = wl.delaunay_graph(1200, wl.rng(5))
        f, C = wl.graph_field(rp, ci, seed=6), 4
        f["color_seed"] = 5
    T, burn = 40, 15
    with g.Sampler([f], precision=g.FP64, chains=C, seed=19, burn_in=burn, flags=g.FLAG_NO_RESIDENT) as s:
        m0, v0 = s.fetch_pooled(0)
        assert np.all(m0 == 0) and np.all(np.isnan(v0))  # nothing accumulated yet
        s.sweep(T)
        mean, var = s.fetch_pooled(0)
        per = [s.fetch(0, c) for c in range(C)]
    k = T - burn
    mu, vv = _pooled([p["mean"] for p in per], [p["var"] * (k - 1) for p in per], k)
    assert relerr(mean, mu) <= 1e-12 and relerr(var, vv) <= 1e-10
    # and against the oracle's chains pooled the same way
    st, _ = run_oracle(f, C, T, seed=19, stream=0, burn_in=burn)
    mo, vo = _pooled(st.mean, st.m2, st.count)
    assert relerr(mean, mo) <= 1e-12 and relerr(var, vo) <= 1e-10


def test_fetch_pooled_fp32_volume():
    f = wl.small_lattice(wl.LATTICE3D_6, (40, 40, 48), 8)
    with g.Sampler([f], precision=g.FP32, chains=8, seed=23, burn_in=10, graph_sweeps=10) as s:
        s.sweep(50)
        mean, var = s.fetch_pooled(0)
    st, _ = run_oracle(f, 8, 50, seed=23, stream=0, burn_in=10)
    mo, vo = _pooled(st.mean, st.m2, st.count)
    assert relerr(mean, mo) <= TOL_FP32_1000 and relerr(var, vo) <= 1e-3
