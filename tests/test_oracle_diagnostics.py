"""Pins of the oracle's chain diagnostics (CPU only).

IAT (Geyer's initial monotone sequence) against the closed forms of stationary processes:
AR(1) with coefficient phi has IAT (1 + phi)/(1 - phi); MA(1) with coefficient theta has
IAT 1 + 2 theta/(1 + theta^2); white noise has IAT 1; plus a sequence small enough to work by
hand.  PSRF (Brooks-Gelman form) against chains with identical moments, where it equals
sqrt((N - 1)/N) exactly, and long normal chains with known mean offsets.
"""
import numpy as np
import pytest

import oracle


def _ar1(phi, N, seed):
    g = np.random.default_rng(seed)
    e = g.standard_normal(N + 1000)
    x = np.zeros_like(e)
    for t in range(1, len(e)):
        x[t] = phi * x[t - 1] + e[t]
    return x[1000:]


@pytest.mark.parametrize("phi", [0.5, 0.9])
def test_iat_ar1_closed_form(phi):
    x = _ar1(phi, 400_000, 3)
    want = (1 + phi) / (1 - phi)
    assert abs(oracle.iat(x) / want - 1) < 0.08


@pytest.mark.parametrize("theta", [0.8, -0.5])
def test_iat_ma1_closed_form(theta):
    e = np.random.default_rng(5).standard_normal(400_001)
    x = e[1:] + theta * e[:-1]
    want = 1 + 2 * theta / (1 + theta ** 2)
    assert abs(oracle.iat(x) - want) < 0.05


def test_iat_white_noise():
    x = np.random.default_rng(7).standard_normal(400_000)
    assert abs(oracle.iat(x) - 1.0) < 0.05
    assert oracle.ess(x) == pytest.approx(len(x) / oracle.iat(x))


def test_iat_by_hand():
    # x = 1, -1, 1, ... (N = 10): gamma(k) = (-1)^k (N - k)/N, so every Gamma_m = 1/10 > 0, the
    # monotone sum over m = 0..4 is 1/2 and kappa = -1 + 2 * 1/2 = 0, floored at 1/log10(10) = 1.
    x = np.array([1.0, -1.0] * 5)
    assert oracle.iat(x) == pytest.approx(1.0)
    # x = 0, 0, 1, 1, 0, 0, 1, 1 (N = 8): deviations +-1/2 with signs s = (-,-,+,+,-,-,+,+), so
    # gamma(k) = (1/4)(1/8) sum_t s_t s_{t+k}: gamma(0) = 1/4, gamma(1) = 1/32, gamma(2) = -6/32,
    # gamma(3) = -1/32.  Gamma_0 = 9/32 > 0, Gamma_1 = -7/32 < 0, so M = 0 and
    # kappa = (-1/4 + 2 * 9/32) / (1/4) = 1.25 (above the floor 1/log10(8) = 1.107).
    assert oracle.iat(np.array([0.0, 0.0, 1.0, 1.0] * 2)) == pytest.approx(1.25)
    # x = 0,0,0,0,1,1,0,1,1,2 (N = 10, mean 3/5): gamma(0..5) = 11/25, 31/250, 6/125, -7/250,
    # 9/250, 1/50, so Gamma_0..3 = 141/250, 5/250, 14/250, -57/250 and M = 2; the monotone
    # sequence clips Gamma_2 to 5/250, the sum is 151/250 and kappa = (-110 + 302)/110 = 96/55
    # (1.909 without the monotone step).
    assert oracle.iat(np.array([0, 0, 0, 0, 1, 1, 0, 1, 1, 2], float)) == pytest.approx(96 / 55)
    # N = 4: the same pattern gives 1.5 < 1/log10(4), so the floor applies.
    assert oracle.iat(np.array([0.0, 0.0, 1.0, 1.0])) == pytest.approx(1.0 / np.log10(4.0))
    assert np.isnan(oracle.iat(np.ones(50)))
    assert np.isnan(oracle.iat(np.arange(3.0)))


def test_psrf_identical_moments():
    g = np.random.default_rng(1)
    base = g.standard_normal(500)
    chains = np.stack([g.permutation(base) for _ in range(4)])
    assert oracle.psrf(chains) == pytest.approx(np.sqrt(499 / 500), rel=1e-12)


def test_psrf_mean_offsets():
    g = np.random.default_rng(2)
    mu = np.array([0.0, 0.3, -0.2, 0.5])
    N = 200_000
    chains = mu[:, None] + g.standard_normal((4, N))
    m = len(mu)
    want = np.sqrt((N - 1) / N + (m + 1) / m * np.var(mu, ddof=1))
    assert oracle.psrf(chains) == pytest.approx(want, rel=2e-3)
    same = g.standard_normal((3, N))
    assert oracle.psrf(same) == pytest.approx(1.0, abs=2e-3)


def test_psrf_moments_matches_chains():
    g = np.random.default_rng(4)
    ch = g.standard_normal((3, 1000)) * np.array([[1.0], [1.5], [0.7]]) + np.array([[0.0], [0.1], [0.2]])
    r1 = oracle.psrf(ch)
    r2 = oracle.psrf_moments(ch.mean(1), ch.var(1, ddof=1), 1000)
    assert r1 == pytest.approx(r2, rel=1e-12)
    assert np.isnan(oracle.psrf(ch[:1]))
