"""GPU parity of the generators and of Jones-Plassmann colouring (bit-exact integer work).

- Philox4x32-10 words computed by the CUDA library equal the oracle's, bit for bit.
- The update normals agree with the oracle's FP64 Box-Muller: to rounding in FP64, within the
  single-precision error budget in FP32.
- The GPU's JP colouring equals the oracle's sequential greedy colouring in decreasing
  (priority, index) order, exactly; with priority = n - 1 - index it is the paper's greedy; a
  sampler's own colouring (largest-degree-first priorities, or the random ones on request) too.
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


@pytest.mark.parametrize("seed,c1,c2,c3", [(0, 0, 0, 0), (0xDEADBEEFCAFEF00D, 7, 123456, 3 << 24),
                                           (2**64 - 1, 2**32 - 1, 2**32 - 1, 2**32 - 1)])
def test_philox_words_bit_exact(seed, c1, c2, c3):
    n = 1 << 18
    got = g.philox_words(seed, c1, c2, c3, n)
    want = oracle.philox_fill(seed, c1, c2, c3, n)
    assert np.array_equal(got, want)


def test_philox_words_known_answer():
    # counter (0,0,0,0), key 0 -> published Philox4x32-10 answer
    got = g.philox_words(0, 0, 0, 0, 1)[0]
    assert [hex(v) for v in got] == ["0x6627e8d5", "0xe169c58d", "0xbc57ac4c", "0x9b00dbd8"]


LANE_CHAINS = [(4, 0), (4, 1), (4, 2), (4, 3), (4, 4), (4, 7), (4, 13), (2, 0), (2, 1), (1, 0)]


@pytest.mark.parametrize("lanes,chain", LANE_CHAINS)
def test_site_normals_fp64(lanes, chain):
    n = 1 << 17
    got = g.site_normals(99, 5, 3, chain, n, g.FP64, lanes=lanes)
    want = oracle.site_normals(99, n, 5, 3, chain, lanes)
    assert np.max(np.abs(got - want) / np.maximum(np.abs(want), 1.0)) < 1e-14


@pytest.mark.parametrize("lanes,chain", LANE_CHAINS[:5] + LANE_CHAINS[-3:])
def test_site_normals_fp32(lanes, chain):
    n = 1 << 20
    got = g.site_normals(7, 11, 0, chain, n, g.FP32, lanes=lanes).astype(np.float64)
    want = oracle.site_normals(7, n, 11, 0, chain, lanes)
    # radius and angle each carry a few single-precision ulps; no tail loses relative precision
    assert np.max(np.abs(got - want) / np.maximum(np.abs(want), 1.0)) < 3e-6


def _graphs():
    g0 = wl.rng(5)
    out = {"path": wl.path_graph(50), "cycle_odd": wl.cycle_graph(51), "star": wl.star_graph(3000),
           "grid8": wl.grid_graph(40, 37, eight=True), "er_sparse": wl.random_graph(2000, 0.004, g0),
           "er_dense": wl.random_graph(300, 0.3, g0), "k40": wl.random_graph(40, 1.01, g0),
           "isolated": wl.csr_from_edges(10, np.array([[0, 1], [1, 2], [5, 6]]))}
    rp, ci, _ = wl.delaunay_graph(16384, wl.rng(3))
    out["delaunay16k"] = (rp, ci)
    return out


GRAPHS = _graphs()


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("seed", [1, 0xABCDEF0123])
def test_jp_colouring_bit_exact(name, seed):
    rp, ci = GRAPHS[name]
    colors, k = g.color_graph(rp, ci, seed=seed)
    want, kw = oracle.color_graph(rp, ci, seed)
    assert np.array_equal(colors, want)
    assert k == kw
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    assert np.all(colors[rows] != colors[ci])


@pytest.mark.parametrize("name", ["path", "grid8", "er_sparse", "delaunay16k", "star"])
def test_jp_with_index_priorities_is_papers_greedy(name):
    rp, ci = GRAPHS[name]
    n = len(rp) - 1
    prio = (n - 1 - np.arange(n)).astype(np.uint32)
    colors, k = g.color_graph(rp, ci, priorities=prio)
    want, kw = oracle.color_greedy(rp, ci, prio)
    assert np.array_equal(colors, want) and k == kw


def test_jp_all_equal_priorities_break_ties_by_index():
    rp, ci = wl.grid_graph(17, 23)
    prio = np.zeros(17 * 23, np.uint32)
    colors, _ = g.color_graph(rp, ci, priorities=prio)
    want, _ = oracle.color_greedy(rp, ci, prio)
    assert np.array_equal(colors, want)


def test_single_vertex_graph():
    colors, k = g.color_graph(np.array([0, 0]), np.zeros(0, np.int32), seed=3)
    assert k == 1 and colors.tolist() == [0]


@pytest.mark.parametrize("name", ["er_sparse", "er_dense", "star", "k40", "isolated", "delaunay16k"])
@pytest.mark.parametrize("random", [False, True])
def test_sampler_colouring_bit_exact(name, random):
    # a sampler's own JP colouring: largest-degree-first priorities by default, the random ones
    # under GMRF_FLAG_COLOR_RANDOM; equal to the oracle's greedy colouring in that order, exactly
    rp, ci = GRAPHS[name]
    f = dict(wl.graph_field(rp, ci, seed=4), color_seed=9)
    flags = g.FLAG_COLOR_RANDOM if random else 0
    with g.Sampler([f], precision=g.FP32, chains=1, seed=1, flags=flags) as s:
        colors, k = s.colors(0)
    want, kw = oracle.color_graph(rp, ci, 9, ldf=not random)
    assert np.array_equal(colors, want) and k == kw


def test_ldf_takes_fewer_colours_on_the_delaunay_benchmark_graph():
    rp, ci = GRAPHS["delaunay16k"]
    f = dict(wl.graph_field(rp, ci, seed=4), color_seed=3)
    ks = []
    for flags in (g.FLAG_COLOR_RANDOM, 0):
        with g.Sampler([f], precision=g.FP32, chains=8, seed=1, flags=flags) as s:
            ks.append(s.colors(0)[1])
    assert ks == [7, 6]


@pytest.mark.parametrize("resident", [True, False])
@pytest.mark.parametrize("random", [False, True])
def test_sampler_colouring_parity(resident, random):
    # sweeps over either colouring (graph resident kernel, or the per-colour path) against the
    # oracle run on the same colouring
    from gmrf_testutil import TOL_FP32_1000, relerr, run_oracle, trace_relerr

    rp, ci, _ = wl.delaunay_graph(3000, wl.rng(12))
    f = dict(wl.graph_field(rp, ci, seed=13), color_seed=14, color_random=random)
    flags = (g.FLAG_COLOR_RANDOM if random else 0) | (0 if resident else g.FLAG_NO_RESIDENT)
    with g.Sampler([f], precision=g.FP32, chains=2, seed=15, flags=flags, burn_in=20) as s:
        s.sweep(60)
        assert (s.info()["resident"] == 2) == resident
        res = [s.fetch(0, c, trace=60) for c in range(2)]
        colors, _ = s.colors(0)
    want, _ = oracle.color_graph(rp, ci, 14, ldf=not random)
    assert np.array_equal(colors, want)
    st, out = run_oracle(f, 2, 60, seed=15, stream=0, burn_in=20)
    for c in range(2):
        assert relerr(res[c]["x"], st.x[c]) <= TOL_FP32_1000
        assert relerr(res[c]["mean"], st.mean[c]) <= TOL_FP32_1000
        assert trace_relerr(res[c]["tau_trace"], out["tau_trace"][c]) <= TOL_FP32_1000
