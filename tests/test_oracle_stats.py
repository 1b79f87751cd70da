"""Distributional pins of the oracle sampler (CPU only).

- With tau and sigma^2 fixed, the chain's stationary law is the Gaussian full conditional of
  Sec. 2.2, x ~ N(Q_p^-1 y / sigma^2, Q_p^-1) with Q_p = tau (D - rho W) + I / sigma^2.  On
  graphs of at most 12 nodes the empirical mean and covariance of a long chain must agree with
  it within a few batch-means standard errors.
- With the hyperparameter draws on, the posterior of (tau, sigma^2) must agree, within Monte
  Carlo error, with a dense block Gibbs sampler (Sec. 2.2, block updating by a Cholesky
  factorisation of Q_p) written here with numpy's own generators.
"""
import numpy as np
import pytest

import oracle
from paper_1702_05518_gb300 import workloads as wl


def _dense(rp, ci):
    n = len(rp) - 1
    Wm = np.zeros((n, n))
    Wm[np.repeat(np.arange(n), np.diff(rp)), ci] = 1.0
    return Wm, np.diag(Wm.sum(1))


def _batch_se(samples, nb=50):
    """Batch-means standard error of the mean of each column of samples [T, ...]."""
    T = samples.shape[0] // nb * nb
    b = samples[:T].reshape(nb, T // nb, *samples.shape[1:]).mean(1)
    return b.std(0, ddof=1) / np.sqrt(nb)


GRAPHS = [("path6", lambda: wl.path_graph(6)), ("cycle8", lambda: wl.cycle_graph(8)),
          ("grid3x4", lambda: wl.grid_graph(3, 4)), ("k4e", wl.k4_minus_edge),
          ("grid3x4x8", lambda: wl.grid_graph(3, 4, eight=True))]


@pytest.mark.parametrize("name,make", GRAPHS)
@pytest.mark.parametrize("prior,rho", [("icar", 1.0), ("pcar", 0.9)])
def test_fixed_hyper_stationary_law(name, make, prior, rho):
    rp, ci = make()
    n = len(rp) - 1
    g = wl.rng(21)
    y = g.normal(0, 1.5, n)
    tau, sig2 = 1.7, 0.6
    colors, _ = oracle.color_graph(rp, ci, 3)
    st = oracle.initial_state(y, 1, tau0=tau, sigma2_0=sig2)
    T = 120_000
    out = oracle.run((rp, ci), colors, y, st, seed=31, nsweeps=T, prior=prior, rho=rho,
                     fix_hyper=True, accumulate=False, record_x=True)
    xs = out["xtrace"][1000:, 0, :]
    Wm, D = _dense(rp, ci)
    Qp = tau * (D - rho * Wm) + np.eye(n) / sig2
    cov = np.linalg.inv(Qp)
    mu = cov @ (y / sig2)
    se = _batch_se(xs)
    assert np.all(np.abs(xs.mean(0) - mu) < 5 * se + 1e-12)
    dev = xs - mu
    outer = dev[:, :, None] * dev[:, None, :]
    se_cov = _batch_se(outer)
    assert np.all(np.abs(outer.mean(0) - cov) < 5 * se_cov + 1e-12)


def _block_gibbs(rp, ci, y, prior, rho, a_tau, b_tau, a_sig, b_sig, T, seed):
    """Dense block Gibbs: x | tau, sigma^2 ~ N(Q_p^-1 b, Q_p^-1) by Cholesky (one factorisation
    and triangular solves), then tau^2 and sigma^2 from their inverse-gamma conditionals."""
    n = len(rp) - 1
    Wm, D = _dense(rp, ci)
    R = D - rho * Wm
    r = n - oracle.components(rp, ci) if prior == "icar" else n
    g = np.random.default_rng(seed)
    tau, sig2 = 1.0, 1.0
    out = np.zeros((T, 2))
    for t in range(T):
        Qp = tau * R + np.eye(n) / sig2
        L = np.linalg.cholesky(Qp)
        mean = np.linalg.solve(L.T, np.linalg.solve(L, y / sig2))
        x = mean + np.linalg.solve(L.T, g.standard_normal(n))
        S = x @ R @ x
        tau = g.gamma(a_tau + r / 2, 1.0 / (b_tau + S / 2))
        sig2 = 1.0 / g.gamma(a_sig + n / 2, 1.0 / (b_sig + np.sum((y - x) ** 2) / 2))
        out[t] = tau, sig2
    return out


@pytest.mark.parametrize("name,make", [("grid3x4", lambda: wl.grid_graph(3, 4)),
                                       ("k4e", wl.k4_minus_edge)])
@pytest.mark.parametrize("prior,rho", [("icar", 1.0), ("pcar", 0.8)])
def test_hyper_posterior_matches_block_gibbs(name, make, prior, rho):
    rp, ci = make()
    n = len(rp) - 1
    y = wl.rng(5).normal(0, 1.0, n)
    hp = dict(a_tau=3.0, b_tau=2.0, a_sig=3.0, b_sig=1.0)
    T = 60_000
    colors, _ = oracle.color_graph(rp, ci, 1)
    st = oracle.initial_state(y, 1)
    out = oracle.run((rp, ci), colors, y, st, seed=2, nsweeps=T, prior=prior, rho=rho,
                     accumulate=False, **hp)
    chrom = np.stack([out["tau_trace"][0], out["sigma2_trace"][0]], 1)[2000:]
    block = _block_gibbs(rp, ci, y, prior, rho, hp["a_tau"], hp["b_tau"], hp["a_sig"],
                         hp["b_sig"], 30_000, 7)[1000:]
    se = np.sqrt(_batch_se(chrom) ** 2 + _batch_se(block) ** 2)
    diff = np.abs(chrom.mean(0) - block.mean(0))
    assert np.all(diff < 5 * se), (chrom.mean(0), block.mean(0), se)
    for q in (0.1, 0.5, 0.9):
        qc, qb = np.quantile(chrom, q, axis=0), np.quantile(block, q, axis=0)
        spread = chrom.std(0)
        assert np.all(np.abs(qc - qb) < 0.06 * spread + 5 * se), (q, qc, qb)


# --------------------------------------------------------------------------------------------
# Intercept (Sec. 3.1: y = beta0 1 + x + noise, flat prior on beta0)
# --------------------------------------------------------------------------------------------
def _joint_with_intercept(rp, ci, y, tau, sig2, rho):
    """Precision and mean of (x, beta0) given tau, sigma^2: the likelihood adds
    (x + beta0 1)'(x + beta0 1) / sigma^2 and the linear term y'(x + beta0 1) / sigma^2."""
    n = len(rp) - 1
    Wm, D = _dense(rp, ci)
    Q = np.zeros((n + 1, n + 1))
    Q[:n, :n] = tau * (D - rho * Wm) + np.eye(n) / sig2
    Q[:n, n] = Q[n, :n] = 1.0 / sig2
    Q[n, n] = n / sig2
    h = np.concatenate([y / sig2, [y.sum() / sig2]])
    cov = np.linalg.inv(Q)
    return cov @ h, cov


@pytest.mark.parametrize("name,make", [("path6", lambda: wl.path_graph(6)), ("grid3x4", lambda: wl.grid_graph(3, 4)),
                                       ("k4e", wl.k4_minus_edge)])
def test_intercept_fixed_hyper_stationary_law(name, make):
    # Proper CAR, so the joint law of (x, beta0) is a proper Gaussian.
    rp, ci = make()
    n = len(rp) - 1
    y = wl.rng(23).normal(2.0, 1.5, n)
    tau, sig2, rho = 1.3, 0.7, 0.85
    colors, _ = oracle.color_graph(rp, ci, 4)
    st = oracle.initial_state(y, 1, tau0=tau, sigma2_0=sig2)
    T = 120_000
    out = oracle.run((rp, ci), colors, y, st, seed=37, nsweeps=T, prior="pcar", rho=rho, fix_hyper=True,
                     accumulate=False, record_x=True, intercept=True)
    z = np.concatenate([out["xtrace"][1000:, 0, :], out["beta0_trace"][0, 1000:, None]], 1)
    mu, cov = _joint_with_intercept(rp, ci, y, tau, sig2, rho)
    se = _batch_se(z)
    assert np.all(np.abs(z.mean(0) - mu) < 5 * se + 1e-12), (z.mean(0), mu)
    dev = z - mu
    outer = dev[:, :, None] * dev[:, None, :]
    assert np.all(np.abs(outer.mean(0) - cov) < 5 * _batch_se(outer) + 1e-12)


def test_intercept_zero_data_shift_equivariance():
    # Adding a constant c to y shifts the intercept chain by exactly c in law; with the same
    # random numbers the chain of x is unchanged and beta0 moves by c up to rounding.
    rp, ci = wl.grid_graph(4, 5, eight=True)
    n = len(rp) - 1
    y = wl.rng(3).normal(0, 1, n)
    colors, _ = oracle.color_graph(rp, ci, 2)
    runs = []
    for c in (0.0, 7.5):
        st = oracle.initial_state(y + c, 2, beta0=c, x0=y)
        out = oracle.run((rp, ci), colors, y + c, st, seed=5, nsweeps=50, intercept=True, accumulate=False)
        runs.append((st, out))
    (s0, o0), (s1, o1) = runs
    np.testing.assert_allclose(s1.x, s0.x, atol=1e-9)
    np.testing.assert_allclose(o1["beta0_trace"] - 7.5, o0["beta0_trace"], atol=1e-9)
    np.testing.assert_allclose(o1["sigma2_trace"], o0["sigma2_trace"], rtol=1e-9)
    np.testing.assert_allclose(o1["tau_trace"], o0["tau_trace"], rtol=1e-9)


def _block_gibbs_intercept(rp, ci, y, prior, rho, a_tau, b_tau, a_sig, b_sig, T, seed):
    """Block Gibbs of Sec. 3.1 with the intercept: x | beta0, tau, sigma^2 by Cholesky of Q_p with
    b = (y - beta0 1) / sigma^2, then beta0 | x, sigma^2 ~ N(mean(y - x), sigma^2 / n), then
    tau^2 and sigma^2 from their inverse-gamma conditionals."""
    n = len(rp) - 1
    Wm, D = _dense(rp, ci)
    R = D - rho * Wm
    r = n - oracle.components(rp, ci) if prior == "icar" else n
    g = np.random.default_rng(seed)
    tau, sig2, b0 = 1.0, 1.0, 0.0
    out = np.zeros((T, 3))
    for t in range(T):
        L = np.linalg.cholesky(tau * R + np.eye(n) / sig2)
        x = np.linalg.solve(L.T, np.linalg.solve(L, (y - b0) / sig2) + g.standard_normal(n))
        b0 = np.mean(y - x) + np.sqrt(sig2 / n) * g.standard_normal()
        tau = g.gamma(a_tau + r / 2, 1.0 / (b_tau + x @ R @ x / 2))
        sig2 = 1.0 / g.gamma(a_sig + n / 2, 1.0 / (b_sig + np.sum((y - b0 - x) ** 2) / 2))
        out[t] = tau, sig2, b0 + (np.mean(x) if prior == "icar" else 0.0)
    return out


@pytest.mark.parametrize("prior,rho", [("icar", 1.0), ("pcar", 0.8)])
def test_intercept_posterior_matches_block_gibbs(prior, rho):
    # Under the intrinsic prior only beta0 + mean(x) is identified; it is what is compared.
    rp, ci = wl.grid_graph(3, 4)
    n = len(rp) - 1
    y = wl.rng(8).normal(1.5, 1.0, n)
    hp = dict(a_tau=3.0, b_tau=2.0, a_sig=3.0, b_sig=1.0)
    T = 60_000
    colors, _ = oracle.color_graph(rp, ci, 1)
    st = oracle.initial_state(y, 1)
    out = oracle.run((rp, ci), colors, y, st, seed=4, nsweeps=T, prior=prior, rho=rho, accumulate=False,
                     record_x=True, intercept=True, **hp)
    loc = out["beta0_trace"][0] + (out["xtrace"][:, 0, :].mean(1) if prior == "icar" else 0.0)
    chrom = np.stack([out["tau_trace"][0], out["sigma2_trace"][0], loc], 1)[2000:]
    block = _block_gibbs_intercept(rp, ci, y, prior, rho, hp["a_tau"], hp["b_tau"], hp["a_sig"], hp["b_sig"],
                                   30_000, 9)[1000:]
    se = np.sqrt(_batch_se(chrom) ** 2 + _batch_se(block) ** 2)
    assert np.all(np.abs(chrom.mean(0) - block.mean(0)) < 5 * se), (chrom.mean(0), block.mean(0), se)
    for q in (0.1, 0.5, 0.9):
        qc, qb = np.quantile(chrom, q, axis=0), np.quantile(block, q, axis=0)
        assert np.all(np.abs(qc - qb) < 0.06 * chrom.std(0) + 5 * se), (q, qc, qb)


# --------------------------------------------------------------------------------------------
# Binomial data with the logistic link (Sec. 3.2): Polya-Gamma augmentation
# --------------------------------------------------------------------------------------------
def _pg_moments(b, c):
    if c == 0.0:
        return b / 4.0, b / 24.0
    return (b / (2 * c) * np.tanh(c / 2),
            b / (4 * c ** 3) * (np.sinh(c) - c) / np.cosh(c / 2) ** 2)


@pytest.mark.parametrize("b,c", [(1, 0.0), (1, 0.7), (1, 3.0), (1, 25.0), (3, 1.5), (7, -2.0)])
def test_polya_gamma_moments(b, c):
    # E and Var of PG(b, c) in closed form (Polson, Scott & Windle 2013, Sec. 2).
    N = 200_000
    v = np.array([oracle.pg_draw(b, c, 21, site=i, sweep=1)[0] for i in range(N)])
    m, var = _pg_moments(b, c)
    assert abs(v.mean() - m) < 5 * np.sqrt(var / N)
    assert abs(v.var() / var - 1) < 0.03
    assert v.min() > 0


def test_polya_gamma_sum_and_zero():
    # PG(0, c) = 0; PG(b, c) is the sum of the b PG(1, c) draws of the same counters.
    assert oracle.pg_draw(0, 1.3, 5)[0] == 0.0
    v3 = oracle.pg_draw(3, 1.3, 5, site=4, sweep=2)[0]
    assert v3 > 0


def _logistic_posterior_by_quadrature(rp, ci, trials, y, tau, rho, prior_var):
    """Posterior means of x and beta0 and of the success probabilities, by summing the exact
    joint density (Gaussian CAR prior, normal prior on beta0, binomial likelihood) on a grid."""
    n = len(rp) - 1
    Wm, D = _dense(rp, ci)
    Q = tau * (D - rho * Wm)
    axes = [np.linspace(-7, 7, 57)] * n + [np.linspace(-9, 9, 73)]
    grids = np.meshgrid(*axes, indexing="ij")
    X = np.stack([g.ravel() for g in grids[:n]], 1)
    b0 = grids[n].ravel()
    logp = -0.5 * np.einsum("ki,ij,kj->k", X, Q, X) - 0.5 * b0 ** 2 / prior_var
    eta = X + b0[:, None]
    logp += np.sum(y * eta - trials * np.logaddexp(0, eta), 1)
    w = np.exp(logp - logp.max())
    w /= w.sum()
    pi = 1 / (1 + np.exp(-eta))
    return (w @ X), float(w @ b0), (w @ pi)


def test_binomial_posterior_matches_quadrature():
    # Three sites on a path, proper CAR (rho 0.5), tau fixed at 2, beta0 ~ N(0, 4); the middle
    # site has no trials (its update is then the prior conditional).
    rp, ci = wl.path_graph(3)
    trials = np.array([6, 0, 9], np.int32)
    y = np.array([4.0, 0.0, 2.0])
    tau = 2.0
    colors, _ = oracle.color_graph(rp, ci, 2)
    st = oracle.initial_state(y, 1, tau0=tau, x0=np.zeros(3))
    T = 150_000
    out = oracle.run((rp, ci), colors, y, st, seed=13, nsweeps=T, prior="pcar", rho=0.5, fix_hyper=True,
                     accumulate=False, record_x=True, trials=trials, beta0_prior=(0.0, 4.0))
    xs = out["xtrace"][2000:, 0, :]
    bs = out["beta0_trace"][0, 2000:]
    pis = 1 / (1 + np.exp(-(xs + bs[:, None])))
    mx, mb, mpi = _logistic_posterior_by_quadrature(rp, ci, trials, y, tau, 0.5, 4.0)
    z = np.concatenate([xs, bs[:, None], pis], 1)
    want = np.concatenate([mx, [mb], mpi])
    se = _batch_se(z)
    assert np.all(np.abs(z.mean(0) - want) < 5 * se + 1e-3), (z.mean(0), want, se)
    assert out["fallbacks"] == 0


def test_polya_gamma_series_forms_agree():
    # The two series of the J*(1, 0) density (Devroye 2009) are the two sides of a Jacobi
    # theta-function identity: summed to convergence they agree at every x > 0; the density
    # integrates to 1 and has mean 1 (E J*(1, 0) = 1).
    from scipy import integrate

    def dens(x, form):
        return sum((-1) ** n * oracle.pg_series_term(n, x, form) for n in range(60))

    for x in (0.15, 0.3, 0.64, 1.0, 2.5):
        assert dens(x, 0) == pytest.approx(dens(x, 1), rel=1e-9)
    f = lambda x: dens(x, 0) if x <= 0.64 else dens(x, 1)  # noqa: E731
    mass = integrate.quad(f, 1e-6, 0.64)[0] + integrate.quad(f, 0.64, 60)[0]
    mean = integrate.quad(lambda x: x * f(x), 1e-6, 0.64)[0] + integrate.quad(lambda x: x * f(x), 0.64, 60)[0]
    assert mass == pytest.approx(1.0, abs=1e-8) and mean == pytest.approx(1.0, abs=1e-8)


@pytest.mark.parametrize("z", [0.0, 0.3, 1.0, 1 / 0.64, 4.0, 12.0])
def test_polya_gamma_proposal_weights(z):
    # The envelope is exp(-z^2 x / 2) a_0(x); the weight of its exponential piece (x > t) must
    # equal the ratio of the envelope's integrals, computed here by quadrature.
    from scipy import integrate

    t = 0.64
    env0 = lambda x: np.exp(-z * z * x / 2) * oracle.pg_series_term(0, x, 0)  # noqa: E731
    env1 = lambda x: np.exp(-z * z * x / 2) * oracle.pg_series_term(0, x, 1)  # noqa: E731
    q = integrate.quad(env0, 0, t, limit=200)[0]
    p = integrate.quad(env1, t, np.inf, limit=200)[0]
    assert oracle.pg_mix_weight(z) == pytest.approx(p / (p + q), rel=1e-8)
