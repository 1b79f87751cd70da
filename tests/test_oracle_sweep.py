"""Pins of the oracle's sweep, reductions and hyperparameter draws (CPU only).

The expected values here are derived another way than the oracle computes them:
- one sweep: Gaussian conditionals x_i | x_-i read off the dense joint precision
  Q_p = tau (D - rho W) + I / sigma^2 and b = y / sigma^2 (Sec. 2.2: x ~ N(Q_p^-1 b, Q_p^-1)),
  taken colour class by colour class (Algorithm 1);
- the paper's own variance-form local characteristics (Sec. 3.1) in a pure-Python
  single-site sampler, with its own Philox and Box-Muller;
- x'(D - rho W)x as a dense quadratic form;
- Welford accumulators against numpy mean/var of the recorded chain.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1702_05518_gb300 import workloads as wl


def _dense(rp, ci, weights=None):
    n = len(rp) - 1
    Wm = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(rp))
    Wm[rows, ci] = 1.0 if weights is None else weights
    return Wm, np.diag(Wm.sum(1))


def _sym_weights(rp, ci, g):
    """Random positive symmetric edge weights in CSR order."""
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    w_edge = {}
    w = np.zeros(len(ci))
    for e, (i, j) in enumerate(zip(rows, ci)):
        key = (min(i, j), max(i, j))
        if key not in w_edge:
            w_edge[key] = g.uniform(0.5, 2.0)
        w[e] = w_edge[key]
    return w


CASES = [("path", lambda: wl.path_graph(7)), ("cycle", lambda: wl.cycle_graph(8)),
         ("k4e", wl.k4_minus_edge), ("grid4", lambda: wl.grid_graph(3, 4)),
         ("grid8", lambda: wl.grid_graph(3, 4, eight=True)), ("star", lambda: wl.star_graph(6))]


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("prior,rho", [("icar", 1.0), ("pcar", 0.9)])
@pytest.mark.parametrize("weighted", [False, True])
def test_one_sweep_equals_dense_conditionals(name, make, prior, rho, weighted):
    rp, ci = make()
    n = len(rp) - 1
    g = wl.rng(3)
    w = _sym_weights(rp, ci, g) if weighted else None
    y = g.normal(1.0, 1.0, n)
    x0 = g.normal(0.0, 2.0, (2, n))
    tau, sig2 = np.array([2.5, 0.7]), np.array([0.3, 1.7])
    colors, k = oracle.color_graph(rp, ci, seed=17)
    st = oracle.State(x0, tau, sig2)
    seed, sweep, stream = 41, 5, 3
    oracle.run((rp, ci), colors, y, st, seed=seed, nsweeps=1, stream=stream, start_sweep=sweep,
               prior=prior, rho=rho, fix_hyper=True, weights=w)
    Wm, D = _dense(rp, ci, w)
    for c in range(2):
        Qp = tau[c] * (D - rho * Wm) + np.eye(n) / sig2[c]
        b = y / sig2[c]
        x = x0[c].copy()
        for col in range(k):
            idx = np.flatnonzero(colors == col)
            new = {}
            for i in idx:
                cond_mean = (b[i] - (Qp[i] @ x - Qp[i, i] * x[i])) / Qp[i, i]
                z = oracle.site_normal(seed, int(i), sweep, stream, c, oracle.lanes_for(2))
                new[i] = cond_mean + z / math.sqrt(Qp[i, i])
            for i, v in new.items():
                x[i] = v
        np.testing.assert_allclose(st.x[c], x, rtol=1e-12, atol=1e-12)


def test_tau_zero_gives_independent_normals():
    # tau = 0 removes the prior: every site is drawn from N(y_i, sigma^2) independently.
    rp, ci = wl.grid_graph(6, 5)
    n = 30
    y = wl.rng(2).normal(0, 3, n)
    colors, _ = oracle.lattice_colors(oracle.LAT2D_4, (6, 5))
    st = oracle.initial_state(y, 3, tau0=0.0, sigma2_0=[0.25, 1.0, 4.0])
    oracle.run((rp, ci), colors, y, st, seed=8, nsweeps=1, start_sweep=2, fix_hyper=True)
    for c in range(3):
        z = oracle.site_normals(8, n, 2, 0, c, oracle.lanes_for(3))
        np.testing.assert_allclose(st.x[c], y + math.sqrt(st.sigma2[c]) * z, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("prior", ["icar", "pcar"])
def test_colour_class_does_not_read_its_own_old_values(prior):
    # Sites of one colour are conditionally independent given the others (Sec. 2.3): changing
    # the old values of colour 0 changes nothing of a sweep (colour 0 is drawn first), while
    # changing colour 1 does.
    rp, ci = wl.grid_graph(5, 6, eight=True)
    n = 30
    g = wl.rng(4)
    y = g.normal(0, 1, n)
    colors, k = oracle.color_graph(rp, ci, 5)
    x0 = g.normal(0, 1, (1, n))
    base = oracle.State(x0, [1.3], [0.8])
    pert0 = oracle.State(np.where(colors == 0, x0 + 5.0, x0), [1.3], [0.8])
    pert1 = oracle.State(np.where(colors == 1, x0 + 5.0, x0), [1.3], [0.8])
    outs = [oracle.run((rp, ci), colors, y, s, seed=6, nsweeps=1, prior=prior, rho=0.8)
            for s in (base, pert0, pert1)]
    assert np.array_equal(base.x, pert0.x)
    assert np.array_equal(outs[0]["tau_trace"], outs[1]["tau_trace"])
    assert base.tau[0] == pert0.tau[0] and base.sigma2[0] == pert0.sigma2[0]
    assert not np.array_equal(base.x, pert1.x)


def _philox_py(ctr, key):
    c = list(ctr)
    k0, k1 = key
    M = 0xFFFFFFFF
    for _ in range(10):
        p0 = 0xD2511F53 * c[0]
        p1 = 0xCD9E8D57 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k0) & M, p1 & M, ((p0 >> 32) ^ c[3] ^ k1) & M, p0 & M]
        k0 = (k0 + 0x9E3779B9) & M
        k1 = (k1 + 0xBB67AE85) & M
    return c


def _normal_py(seed, site, sweep, stream, chain, lanes):
    G = 4 // lanes
    w = _philox_py([site // G, sweep, stream, chain >> 2], [seed & 0xFFFFFFFF, seed >> 32])
    idx = (site % G) * lanes + chain % lanes
    pair = (w[0], w[1]) if idx < 2 else (w[2], w[3])
    ua, ub = [(v + 0.5) / 2**32 for v in pair]
    r = math.sqrt(-2 * math.log(ua))
    return r * (math.cos(2 * math.pi * ub) if (idx & 1) == 0 else math.sin(2 * math.pi * ub))


@pytest.mark.parametrize("chains", [1, 2, 5])
def test_single_site_sampler_in_colour_order_matches(chains):
    # The paper's single-site sampler (Sec. 3.1, variance form with tau^2 = 1/tau):
    #   mu_i = s2_i (y_i / sigma^2 + sum_j w_ij x_j / tau^2),  s2_i = tau^2 sigma^2 / (sigma^2 D_ii + tau^2),
    # visiting sites colour class by colour class, equals the chromatic sweep (Sec. 2.3, "single-site
    # sampling is chromatic sampling with k = n", up to the visiting order).
    rp, ci = wl.grid_graph(4, 5, eight=True)
    n = 20
    g = wl.rng(9)
    y = g.normal(0, 1, n)
    colors, k = oracle.color_graph(rp, ci, 21)
    st = oracle.initial_state(y, chains, tau0=np.linspace(0.5, 3, 5)[:chains],
                              sigma2_0=np.linspace(0.2, 2, 5)[:chains])
    x = st.x.copy()
    seed, T = 12345678901, 6
    oracle.run((rp, ci), colors, y, st, seed=seed, nsweeps=T, stream=4, fix_hyper=True,
               accumulate=False)
    deg = np.diff(rp)
    lanes = 1 if chains == 1 else (2 if chains == 2 else 4)
    for c in range(chains):
        tau2, sig2 = 1.0 / np.linspace(0.5, 3, 5)[c], np.linspace(0.2, 2, 5)[c]
        for t in range(T):
            for col in range(k):
                for i in np.flatnonzero(colors == col):
                    s2i = tau2 * sig2 / (sig2 * deg[i] + tau2)
                    mu = s2i * (y[i] / sig2 + x[c, ci[rp[i]:rp[i + 1]]].sum() / tau2)
                    x[c, i] = mu + math.sqrt(s2i) * _normal_py(seed, int(i), t, 4, c, lanes)
    np.testing.assert_allclose(st.x, x, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("rho", [1.0, 0.95, 0.0])
def test_quadform_dense(rho):
    rp, ci, _ = wl.delaunay_graph(120, wl.rng(5))
    g = wl.rng(6)
    x = g.normal(2, 1, 120)
    w = _sym_weights(rp, ci, g)
    for weights in (None, w):
        Wm, D = _dense(rp, ci, weights)
        want = x @ (D - rho * Wm) @ x
        assert oracle.quadform(rp, ci, x, rho, weights) == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("prior,rho", [("icar", 1.0), ("pcar", 0.95)])
def test_hyper_draws_follow_the_conjugate_conditionals(prior, rho):
    # After one sweep tau and sigma^2 are the Gamma variates of the conditionals of Sec. 3.1,
    # written here in the paper's inverse-gamma form: tau^2 | x ~ InvGam(a + r/2, b + x'(D - rho W)x / 2)
    # with r = n - 1 (connected, intrinsic) or n (proper); sigma^2 | x, y ~ InvGam(a + n/2, b + |y - x|^2 / 2).
    rp, ci = wl.grid_graph(5, 5, eight=True)
    n = 25
    g = wl.rng(13)
    y = g.normal(0, 1, n)
    colors, _ = oracle.color_graph(rp, ci, 2)
    st = oracle.initial_state(y, 2, tau0=[1.0, 3.0], sigma2_0=[0.5, 2.0])
    oracle.run((rp, ci), colors, y, st, seed=77, nsweeps=1, start_sweep=9, stream=6, prior=prior,
               rho=rho, a_tau=1.5, b_tau=0.2, a_sig=2.0, b_sig=0.3)
    Wm, D = _dense(rp, ci)
    r = n - 1 if prior == "icar" else n
    for c in range(2):
        x = st.x[c]
        S = x @ (D - rho * Wm) @ x
        R = np.sum((y - x) ** 2)
        g_tau, _ = oracle.gamma_draw(1.5 + r / 2, 1.0, 77, 9, 6, oracle.TAG_TAU, c)
        g_sig, _ = oracle.gamma_draw(2.0 + n / 2, 1.0, 77, 9, 6, oracle.TAG_SIG, c)
        assert 1.0 / st.tau[c] == pytest.approx((0.2 + S / 2) / g_tau, rel=1e-12)
        assert st.sigma2[c] == pytest.approx((0.3 + R / 2) / g_sig, rel=1e-12)


def test_accumulators_match_recorded_chain():
    rp, ci = wl.cycle_graph(9)
    y = wl.rng(1).normal(0, 1, 9)
    colors, _ = oracle.color_graph(rp, ci, 3)
    st = oracle.initial_state(y, 2)
    out = oracle.run((rp, ci), colors, y, st, seed=4, nsweeps=60, burn_in=10, thin=3,
                     record_x=True)
    kept = [t for t in range(60) if t >= 10 and (t - 10) % 3 == 0]
    xs = out["xtrace"][kept]  # [K, C, n]
    assert st.count == len(kept)
    np.testing.assert_allclose(st.mean, xs.mean(0), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(st.m2 / (st.count - 1), xs.var(0, ddof=1), rtol=1e-10, atol=1e-13)


def test_checkpoint_resume_is_exact():
    rp, ci = wl.grid_graph(6, 7)
    y = wl.rng(8).normal(0, 1, 42)
    colors, _ = oracle.lattice_colors(oracle.LAT2D_4, (6, 7))
    a = oracle.initial_state(y, 3)
    oracle.run((rp, ci), colors, y, a, seed=5, nsweeps=40, burn_in=7)
    b = oracle.initial_state(y, 3)
    oracle.run((rp, ci), colors, y, b, seed=5, nsweeps=25, burn_in=7)
    b2 = b.copy()
    oracle.run((rp, ci), colors, y, b2, seed=5, nsweeps=15, start_sweep=25, burn_in=7)
    for f in ("x", "tau", "sigma2", "mean", "m2"):
        assert np.array_equal(getattr(a, f), getattr(b2, f)), f
    assert a.count == b2.count


def test_lattice_graph_run_equals_explicit_grid():
    # The oracle's lattice neighbourhood and an explicit CSR grid give the same chain.
    y = wl.rng(3).normal(0, 1, 35)
    rp1, ci1 = oracle.lattice_csr(oracle.LAT2D_8, (5, 7))
    rp2, ci2 = wl.grid_graph(5, 7, eight=True)
    assert np.array_equal(rp1, rp2) and np.array_equal(ci1, ci2)
    colors, _ = oracle.lattice_colors(oracle.LAT2D_8, (5, 7))
    s1, s2 = oracle.initial_state(y, 1), oracle.initial_state(y, 1)
    oracle.run((rp1, ci1), colors, y, s1, seed=1, nsweeps=5)
    oracle.run((rp2, ci2), colors, y, s2, seed=1, nsweeps=5)
    assert np.array_equal(s1.x, s2.x)
