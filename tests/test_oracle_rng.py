"""Pins of the oracle's random-number generators (CPU only).

Philox4x32-10 is pinned by the published known-answer vectors; the uniform map by its exact
definition at the extreme words; the Box-Muller normals and the Marsaglia-Tsang Gamma variates
by their distributions (moments and Kolmogorov-Smirnov against scipy).
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle


def _kat(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(golden_dir):
    rows = _kat(golden_dir)
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert list(oracle.philox(ctr, key)) == want


def _philox_py(ctr, key):
    # A third, pure-Python statement of Philox4x32-10 (Salmon et al. SC'11): the oracle must
    # agree with it on arbitrary counters, not only on the three published vectors.
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


def test_philox_matches_independent_statement():
    g = np.random.default_rng(11)
    for _ in range(200):
        ctr = [int(v) for v in g.integers(0, 2**32, 4)]
        key = [int(v) for v in g.integers(0, 2**32, 2)]
        assert list(oracle.philox(ctr, key)) == _philox_py(ctr, key)


def test_philox_fill_counter_layout():
    seed = 0x0123456789ABCDEF
    blk = oracle.philox_fill(seed, 7, 8, 9, 5)
    for i in range(5):
        assert list(blk[i]) == _philox_py([i, 7, 8, 9], [seed & 0xFFFFFFFF, seed >> 32])


def test_uniform_map_exact():
    assert oracle.uniform(0) == 0.5 / 2**32
    assert oracle.uniform(2**32 - 1) == (2**32 - 0.5) / 2**32
    assert 0.0 < oracle.uniform(0) and oracle.uniform(2**32 - 1) < 1.0
    assert oracle.uniform(2**31) == 0.5 + 0.5 / 2**32


def test_box_muller_definition_one_block():
    # z0 = sqrt(-2 ln u0) cos(2 pi u1), z1 = ... sin, z2/z3 from (w2, w3).
    w = np.array([123456789, 987654321, 4000000000, 17], dtype=np.uint32)
    u = (w.astype(np.float64) + 0.5) / 2**32
    r0, r2 = np.sqrt(-2 * np.log(u[0])), np.sqrt(-2 * np.log(u[2]))
    want = [r0 * np.cos(2 * np.pi * u[1]), r0 * np.sin(2 * np.pi * u[1]),
            r2 * np.cos(2 * np.pi * u[3]), r2 * np.sin(2 * np.pi * u[3])]
    np.testing.assert_allclose(oracle.normals4(w), want, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_site_normals_distribution(lanes):
    z = oracle.site_normals(seed=5, n=400_000, sweep=3, stream=1, chain=0, lanes=lanes)
    assert abs(z.mean()) < 5 / np.sqrt(len(z))
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / len(z))
    assert abs(stats.kurtosis(z)) < 0.05
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_site_normals_chains_independent():
    # Chains 0..3 share one Philox block (cos/sin of two Box-Muller pairs): check they are
    # uncorrelated and each standard normal; chain 4 starts a new block.
    n = 200_000
    zs = np.stack([oracle.site_normals(9, n, 0, 2, c, 4) for c in range(5)])
    cc = np.corrcoef(zs)
    assert np.max(np.abs(cc - np.eye(5))) < 5 / np.sqrt(n)
    for c in range(5):
        assert stats.kstest(zs[c], "norm").pvalue > 1e-4
    # the counter layout: chain c uses component c mod 4 of block (site, sweep, stream, c // 4)
    blk = oracle.philox_fill(9, 0, 2, (0 << 24) | 1, 3)
    assert np.allclose(zs[4][:3], [oracle.normals4(b)[0] for b in blk], rtol=0, atol=0)


@pytest.mark.parametrize("shape", [0.4, 1.0, 1.5, 7.25, 2049.0])
def test_gamma_distribution(shape):
    rate = 2.5
    N = 40_000
    g = np.array([oracle.gamma_draw(shape, rate, 77, t, 3, 1, 0)[0] for t in range(N)])
    mean, var = shape / rate, shape / rate**2
    assert abs(g.mean() - mean) < 5 * np.sqrt(var / N)
    assert abs(g.var() / var - 1) < 5 * np.sqrt((2 + 6 / shape) / N)
    assert stats.kstest(g, stats.gamma(shape, scale=1 / rate).cdf).pvalue > 1e-4


def test_gamma_counters_and_attempts():
    # Different tags/chains/sweeps give different variates; attempts are counted from 1.
    a, na = oracle.gamma_draw(5.0, 1.0, 1, 0, 0, 1, 0)
    b, nb = oracle.gamma_draw(5.0, 1.0, 1, 0, 0, 2, 0)
    c, nc = oracle.gamma_draw(5.0, 1.0, 1, 0, 0, 1, 1)
    assert len({a, b, c}) == 3 and min(na, nb, nc) >= 1
    # the rate only rescales: same counters, rate 4 -> a / 4 exactly
    a4, _ = oracle.gamma_draw(5.0, 4.0, 1, 0, 0, 1, 0)
    assert a4 == pytest.approx(a / 4.0, rel=1e-15)


def test_lanes_for_chain_counts():
    assert [oracle.lanes_for(c) for c in (1, 2, 3, 4, 5, 8, 64)] == [1, 2, 4, 4, 4, 4, 4]


@pytest.mark.parametrize("lanes", [1, 2])
def test_site_normals_grouped_layout(lanes):
    # With fewer than four chains one Philox block serves G = 4 / lanes consecutive sites:
    # block (site // G, sweep, stream, chain // 4), normal (site % G) * lanes + chain % lanes.
    G = 4 // lanes
    n = 4000
    for chain in range(lanes):
        z = oracle.site_normals(21, n, 7, 5, chain, lanes)
        blk = oracle.philox_fill(21, 7, 5, 0, n // G)
        want = np.array([oracle.normals4(blk[i // G])[(i % G) * lanes + chain] for i in range(n)])
        assert np.array_equal(z, want)
    # every normal of a block is used exactly once, so the draws are independent standard normals
    zs = np.stack([oracle.site_normals(3, 200_000, 0, 0, c, lanes) for c in range(lanes)])
    for c in range(lanes):
        assert stats.kstest(zs[c], "norm").pvalue > 1e-4
        a, b = zs[c][0::2], zs[c][1::2]
        assert abs(np.corrcoef(a, b)[0, 1]) < 5 / np.sqrt(len(a))
