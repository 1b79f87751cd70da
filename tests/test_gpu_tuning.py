"""Launch configurations (gmrf_tuning) and the autotuner: every configuration the knobs allow
keeps parity with the oracle (a configuration changes only the rounding of the partial sums),
invalid ones are rejected, and gmrf_autotune returns a configuration (cached per process) that
samplers accept.
"""
import time

import numpy as np
import pytest

from gmrf_testutil import TOL_FP32_1, TOL_FP64, relerr, run_oracle, trace_relerr
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


def _check(f, C, T, precision, tuning, seed=5, tol=None, **kw):
    with g.Sampler([f], precision=precision, chains=C, seed=seed, tuning=tuning,
                   flags=g.FLAG_NO_RESIDENT, **kw) as s:
        s.sweep(T)
        res = [s.fetch(0, c, trace=T) for c in range(C)]
    st, out = run_oracle(f, C, T, seed=seed, stream=0)
    tol = tol or (TOL_FP32_1 if precision == g.FP32 else TOL_FP64)
    for c in range(C):
        assert relerr(res[c]["x"], st.x[c]) <= tol
        assert trace_relerr(res[c]["tau_trace"], out["tau_trace"][c]) <= tol


@pytest.mark.parametrize("quad", [(1, 0), (2, 0), (3, 0), (4, 0), (5, 0), (-1, 0), (1, 24), (3, 40), (5, 54)])
def test_quad_configurations(quad):
    f = wl.small_lattice(wl.LATTICE2D_8, (130, 200), 3)
    _check(f, 1, 1, g.FP32, {"quad_config": quad[0], "quad_rows": quad[1]})


@pytest.mark.parametrize("shape", [(8, 8, 512), (24, 40, 1024), (48, 80, 512), (130, 16, 1024)])
@pytest.mark.parametrize("kind", [wl.LATTICE2D_4, wl.LATTICE2D_8])
def test_fused_tiles(kind, shape):
    f = wl.small_lattice(kind, (150, 133), 4)
    r, c, nt = shape
    k = 0 if kind == wl.LATTICE2D_4 else 1
    t = {"fused_rows": [r if i == k else 0 for i in range(2)], "fused_cols": [c if i == k else 0 for i in range(2)],
         "fused_threads": [nt if i == k else 0 for i in range(2)]}
    _check(f, 3, 1, g.FP32, t)


@pytest.mark.parametrize("v", [1, 2, 4])
@pytest.mark.parametrize("tile", [0, 256, 16384])
def test_chains_per_thread_and_step_tile(v, tile):
    f = wl.small_lattice(wl.LATTICE3D_6, (9, 10, 11), 5)
    _check(f, 8, 1, g.FP32, {"chains_per_thread": v, "step_tile": tile})


@pytest.mark.parametrize("v", [1, 2])
def test_csr_fp64_tuned(v):
    f = _delaunay(1500, 6)
    _check(f, 4, 20, g.FP64, {"chains_per_thread": v, "step_tile": 256})


@pytest.mark.parametrize("bad", [{"chains_per_thread": 3}, {"chains_per_thread": 4}, {"step_tile": 100},
                                 {"fused_rows": [16, 0], "fused_cols": [0, 0]}, {"fused_threads": [256, 0]},
                                 {"quad_config": 6}, {"quad_rows": 13}, {"quad_config": 4, "quad_rows": 200},
                                 {"fused_rows": [0, 256], "fused_cols": [0, 256]}])
def test_invalid_tunings(bad):
    # 2 chains: chains_per_thread 4 exceeds them; the 256 x 256 tile with FP64 state does not fit
    f8 = wl.small_lattice(wl.LATTICE2D_8, (64, 64), 1)
    f4 = wl.small_lattice(wl.LATTICE2D_4, (64, 64), 1)
    fields = [f8, f4]
    C = 1 if "quad_config" in bad or "quad_rows" in bad else 2
    with pytest.raises(g.GmrfError) as e:
        g.Sampler(fields, chains=C, precision=g.FP64 if "fused_rows" in bad else g.FP32, tuning=bad)
    assert e.value.status == g.E_INVALID


def test_autotune_returns_a_cached_configuration():
    fields = [wl.small_lattice(wl.LATTICE2D_4, (300, 300), 7), _delaunay(3000, 8)]
    kw = dict(precision=g.FP32, chains=2, seed=9, graph_sweeps=10)
    t0 = time.perf_counter()
    with g.Sampler(fields, tuning="auto", autotune_sweeps=10, **kw) as s:
        first = time.perf_counter() - t0
        tuning, us = s.tuning, s.tuning_us_per_sweep
        s.sweep(1)
        res = [s.fetch(fi, c) for fi in range(2) for c in range(2)]
    assert us > 0 and tuning is not None
    t0 = time.perf_counter()
    with g.Sampler(fields, tuning="auto", autotune_sweeps=10, **kw) as s2:
        second = time.perf_counter() - t0
        assert s2.tuning == tuning and s2.tuning_us_per_sweep == us
    assert second < first  # the second call reads the cache
    for fi, f in enumerate(fields):
        st, _ = run_oracle(f, 2, 1, seed=9, stream=fi)
        for c in range(2):
            assert relerr(res[fi * 2 + c]["x"], st.x[c]) <= TOL_FP32_1


@pytest.mark.parametrize("cl", [1, 2, 4, 8, 16])
def test_graph_cluster_sizes(cl):
    # the resident graph kernel with a chosen number of blocks per chain (1 keeps 5000 sites in one
    # block's shares); every size samples as the oracle does
    f = _delaunay(5000, 21)
    with g.Sampler([f], precision=g.FP32, chains=4, seed=9, tuning={"graph_cluster": cl}, graph_sweeps=10) as s:
        s.sweep(20)
        res = [s.fetch(0, c, trace=20) for c in range(4)]
        info = s.info()
    st, out = run_oracle(f, 4, 20, seed=9, stream=0)
    for c in range(4):
        assert relerr(res[c]["x"], st.x[c]) <= 1e-4
        assert trace_relerr(res[c]["tau_trace"], out["tau_trace"][c]) <= 1e-4
    assert info["wait_timeouts"] == 0


@pytest.mark.parametrize("bad", [{"graph_cluster": 3}, {"graph_cluster": 32}])
def test_invalid_graph_cluster(bad):
    f = _delaunay(1000, 22)
    with pytest.raises(g.GmrfError):
        g.Sampler([f], precision=g.FP32, chains=2, seed=1, tuning=bad)
