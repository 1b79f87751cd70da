"""GPU parity of the chromatic sampler against the oracle, through the C ABI.

Same seeded inputs, same Philox counters: the GPU chain and the oracle chain are coupled draw
for draw, so they are compared element by element with the parity metric
|x_gpu - x_oracle| / max(|x_oracle|, 1):
  FP32 state: <= 1e-5 after one sweep, <= 1e-4 after 1000 coupled sweeps;
  FP64 state: <= 1e-12.
tau and sigma^2 traces are compared with the same bounds, relative to the oracle's value.
Shapes span several tiles with ragged tails (odd extents, padded chain counts).
"""
import numpy as np
import pytest

import oracle
from gmrf_testutil import (TOL_FP32_1, TOL_FP32_1000, TOL_FP64, relerr, run_oracle, trace_relerr,
                           oracle_colors)
from paper_1702_05518_gb300 import gmrf as g
from paper_1702_05518_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1702_05518_gb300 import build

    build.build()


def gpu_run(fields, chains, nsweeps, precision, seed, **kw):
    with g.Sampler(fields, precision=precision, chains=chains, seed=seed, **kw) as s:
        s.sweep(nsweeps)
        res = [[s.fetch(f, c, trace=nsweeps) for c in range(chains)] for f in range(len(fields))]
        info = s.info()
    return res, info


def compare(field, res_f, chains, nsweeps, seed, stream, tol, tol_trace=None, **okw):
    st, out = run_oracle(field, chains, nsweeps, seed=seed, stream=stream, **okw)
    worst_x, worst_t = 0.0, 0.0
    for c in range(chains):
        worst_x = max(worst_x, relerr(res_f[c]["x"], st.x[c]))
        worst_t = max(worst_t, trace_relerr(res_f[c]["tau_trace"], out["tau_trace"][c]),
                      trace_relerr(res_f[c]["sigma2_trace"], out["sigma2_trace"][c]))
    assert worst_x <= tol, f"x parity {worst_x:.3e} > {tol:.1e}"
    assert worst_t <= (tol_trace or tol), f"trace parity {worst_t:.3e}"
    return st, out


def _delaunay(npts, seed, prior_tau=None):
    rp, ci, _ = wl.delaunay_graph(npts, wl.rng(seed))
    f = wl.graph_field(rp, ci, seed=seed + 100)
    f["color_seed"] = seed
    return f


def _weights(field, seed):
    """Symmetric positive weights in [0.5, 2): a hash of the unordered edge {i, j}."""
    rp, ci = field["row_ptr"], field["col_idx"]
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    lo, hi = np.minimum(rows, ci).astype(np.int64), np.maximum(rows, ci).astype(np.int64)
    key = (lo * 1000003 + hi * 7919 + seed) % 999983
    return 0.5 + 1.5 * key / 999983.0


# --------------------------------------------------------------------------------------------
# The 64 x 64 block-image workload (4-neighbour ICAR, checkerboard, FP64, 1000 sweeps, seed 0)
# --------------------------------------------------------------------------------------------
def test_image64_fp64_1000_sweeps():
    f = wl.image_64_block(seed=0)[0]
    res, info = gpu_run([f], 1, 1000, g.FP64, seed=0, burn_in=500, graph_sweeps=16)
    st, out = compare(f, res[0], 1, 1000, 0, 0, TOL_FP64, burn_in=500)
    assert relerr(res[0][0]["mean"], st.mean[0]) <= TOL_FP64
    assert relerr(res[0][0]["var"], st.m2[0] / (st.count - 1)) <= 1e-10
    assert info["sweeps_done"] == 1000 and info["accumulated"] == 500
    assert info["hyper_fallbacks"] == 0


# --------------------------------------------------------------------------------------------
# FP32, one sweep
# --------------------------------------------------------------------------------------------
ONE_SWEEP_CASES = [
    ("2d4_37x53_c1", lambda: wl.small_lattice(wl.LATTICE2D_4, (37, 53), 1), 1, {}),
    ("2d4_37x53_c3", lambda: wl.small_lattice(wl.LATTICE2D_4, (37, 53), 1), 3, {}),
    ("2d4_70x129_c8", lambda: wl.small_lattice(wl.LATTICE2D_4, (70, 129), 2), 8, {}),
    ("2d8_41x30_c1", lambda: wl.small_lattice(wl.LATTICE2D_8, (41, 30), 3), 1, {}),
    ("2d8_101x67_c8", lambda: wl.small_lattice(wl.LATTICE2D_8, (101, 67), 3), 8, {}),
    ("3d6_9x10x11_c2", lambda: wl.small_lattice(wl.LATTICE3D_6, (9, 10, 11), 4), 2, {}),
    ("3d6_17x12x33_c8", lambda: wl.small_lattice(wl.LATTICE3D_6, (17, 12, 33), 4), 8, {}),
    ("csr_3000_c8_pcar", lambda: _delaunay(3000, 5), 8, {"prior": "pcar", "rho": 0.95}),
    ("csr_2500_c5", lambda: _delaunay(2500, 6), 5, {}),
]


@pytest.mark.parametrize("name,make,chains,mk", ONE_SWEEP_CASES, ids=[c[0] for c in ONE_SWEEP_CASES])
def test_fp32_one_sweep(name, make, chains, mk):
    f = make()
    prior = g.PRIOR_PCAR if mk.get("prior") == "pcar" else g.PRIOR_ICAR
    res, _ = gpu_run([f], chains, 1, g.FP32, seed=17, prior=prior, rho=mk.get("rho", 1.0))
    compare(f, res[0], chains, 1, 17, 0, TOL_FP32_1, **mk)


# --------------------------------------------------------------------------------------------
# FP32, 1000 coupled sweeps
# --------------------------------------------------------------------------------------------
LONG_CASES = [
    ("2d8_64x48_c1", lambda: wl.small_lattice(wl.LATTICE2D_8, (64, 48), 7), 1, {}),
    ("2d4_50x45_c4", lambda: wl.small_lattice(wl.LATTICE2D_4, (50, 45), 8), 4, {}),
    ("3d6_12x13x14_c8", lambda: wl.small_lattice(wl.LATTICE3D_6, (12, 13, 14), 9), 8, {}),
    ("csr_1500_c4_pcar", lambda: _delaunay(1500, 10), 4, {"prior": "pcar", "rho": 0.95}),
]


@pytest.mark.parametrize("name,make,chains,mk", LONG_CASES, ids=[c[0] for c in LONG_CASES])
def test_fp32_1000_sweeps(name, make, chains, mk):
    f = make()
    prior = g.PRIOR_PCAR if mk.get("prior") == "pcar" else g.PRIOR_ICAR
    res, info = gpu_run([f], chains, 1000, g.FP32, seed=23, prior=prior, rho=mk.get("rho", 1.0),
                        graph_sweeps=10, burn_in=200)
    st, out = compare(f, res[0], chains, 1000, 23, 0, TOL_FP32_1000, burn_in=200, **mk)
    for c in range(chains):
        assert relerr(res[0][c]["mean"], st.mean[c]) <= TOL_FP32_1000
    assert info["hyper_fallbacks"] == 0


# --------------------------------------------------------------------------------------------
# FP64 on every field kind, weights, several chains
# --------------------------------------------------------------------------------------------
def _weighted_delaunay():
    f = _delaunay(1200, 12)
    f["weights"] = _weights(f, 3)
    return f


FP64_CASES = [
    ("2d8_33x47_c2", lambda: wl.small_lattice(wl.LATTICE2D_8, (33, 47), 11), 2, {}),
    ("3d6_7x9x10_c3", lambda: wl.small_lattice(wl.LATTICE3D_6, (7, 9, 10), 12), 3, {}),
    ("csr_weighted_c2", _weighted_delaunay, 2, {}),
    ("csr_weighted_pcar_c1", _weighted_delaunay, 1, {"prior": "pcar", "rho": 0.8}),
]


@pytest.mark.parametrize("name,make,chains,mk", FP64_CASES, ids=[c[0] for c in FP64_CASES])
def test_fp64_200_sweeps(name, make, chains, mk):
    f = make()
    prior = g.PRIOR_PCAR if mk.get("prior") == "pcar" else g.PRIOR_ICAR
    res, _ = gpu_run([f], chains, 200, g.FP64, seed=29, prior=prior, rho=mk.get("rho", 1.0))
    compare(f, res[0], chains, 200, 29, 0, TOL_FP64, **mk)


def test_weighted_csr_fp32():
    f = _weighted_delaunay()
    res, _ = gpu_run([f], 4, 1, g.FP32, seed=31)
    compare(f, res[0], 4, 1, 31, 0, TOL_FP32_1)


# --------------------------------------------------------------------------------------------
# Batching, graphs, resume, accumulators, plain sweep, extra hyper draw
# --------------------------------------------------------------------------------------------
def _batch():
    return [wl.small_lattice(wl.LATTICE2D_4, (33, 40), 1), _delaunay(700, 2),
            wl.small_lattice(wl.LATTICE3D_6, (5, 6, 7), 3), wl.small_lattice(wl.LATTICE2D_8, (9, 8), 4),
            _delaunay(64, 5)]


@pytest.mark.parametrize("precision", [g.FP32, g.FP64])
def test_batched_equals_single_fields_and_oracle(precision):
    fields = _batch()
    T, C = 12, 2
    res, _ = gpu_run(fields, C, T, precision, seed=41, graph_sweeps=5)
    for fi, f in enumerate(fields):
        # the per-sweep kernels on one field with the batch's launch configuration (a small single
        # 2-D lattice would take the resident path, a lone graph fewer chains per thread: equal
        # to these up to rounding only)
        single, _ = gpu_run([dict(f, stream_id=fi)], C, T, precision, seed=41, flags=g.FLAG_NO_RESIDENT,
                            tuning={"chains_per_thread": 2})
        for c in range(C):
            assert np.array_equal(single[0][c]["x"], res[fi][c]["x"])
            assert np.array_equal(single[0][c]["tau_trace"], res[fi][c]["tau_trace"])
        compare(f, res[fi], C, T, 41, fi, TOL_FP32_1000 if precision == g.FP32 else TOL_FP64)


def test_graph_replay_equals_direct_launches():
    fields = _batch()
    a, _ = gpu_run(fields, 3, 21, g.FP32, seed=43, graph_sweeps=8)
    b, _ = gpu_run(fields, 3, 21, g.FP32, seed=43, graph_sweeps=0)
    for fi in range(len(fields)):
        for c in range(3):
            assert np.array_equal(a[fi][c]["x"], b[fi][c]["x"])
            assert np.array_equal(a[fi][c]["sigma2_trace"], b[fi][c]["sigma2_trace"])


@pytest.mark.parametrize("precision", [g.FP32, g.FP64])
def test_resume_from_fetched_state_is_exact(precision):
    f = wl.small_lattice(wl.LATTICE2D_8, (30, 31), 5)
    C = 2
    full, _ = gpu_run([f], C, 30, precision, seed=47)
    with g.Sampler([f], precision=precision, chains=C, seed=47) as s:
        s.sweep(12)
        part = [s.fetch(0, c) for c in range(C)]
    f2 = dict(f, x0=np.stack([p["x"] for p in part]), tau0=np.array([p["tau"] for p in part]),
              sigma2_0=np.array([p["sigma2"] for p in part]))
    res, _ = gpu_run([f2], C, 18, precision, seed=47, start_sweep=12)
    for c in range(C):
        assert np.array_equal(res[0][c]["x"], full[0][c]["x"])
        assert np.array_equal(res[0][c]["tau_trace"], full[0][c]["tau_trace"][-18:])


def test_accumulators_fp64():
    f = _delaunay(900, 14)
    T = 60
    res, info = gpu_run([f], 2, T, g.FP64, seed=53, burn_in=5, thin=3)
    st, _ = run_oracle(f, 2, T, seed=53, stream=0, burn_in=5, thin=3)
    assert info["accumulated"] == st.count
    for c in range(2):
        assert relerr(res[0][c]["mean"], st.mean[c]) <= TOL_FP64
        assert relerr(res[0][c]["var"], st.m2[c] / (st.count - 1)) <= 1e-10


@pytest.mark.parametrize("kind", ["2d8", "csr"])
def test_plain_fp64_sweep_matches_oracle(kind):
    f = wl.small_lattice(wl.LATTICE2D_8, (50, 61), 6) if kind == "2d8" else _delaunay(2000, 15)
    res, info = gpu_run([f], 2, 60, g.FP64, seed=59, algorithm=g.ALGO_PLAIN, graph_sweeps=7)
    compare(f, res[0], 2, 60, 59, 0, TOL_FP64)
    assert info["sweeps_done"] == 60


def test_extra_hyper_draw():
    f = _delaunay(800, 16)
    C = 2
    x0 = wl.rng(1).normal(0, 1, (C, f["n"]))
    f = dict(f, x0=x0)
    with g.Sampler([f], precision=g.FP64, chains=C, seed=61, a_tau=2.0, b_tau=0.5, a_sigma=3.0,
                   b_sigma=0.25) as s:
        s.hyper_update()
        s.hyper_update()
        got = [s.fetch(0, c) for c in range(C)]
    rank = f["n"] - oracle.components(f["row_ptr"], f["col_idx"])
    for c in range(C):
        S = oracle.quadform(f["row_ptr"], f["col_idx"], x0[c])
        R = float(np.sum((f["y"] - x0[c]) ** 2))
        tau, _ = oracle.gamma_draw(2.0 + rank / 2, 0.5 + S / 2, 61, 1, 0, 5, c)
        prec, _ = oracle.gamma_draw(3.0 + f["n"] / 2, 0.25 + R / 2, 61, 1, 0, 6, c)
        assert got[c]["tau"] == pytest.approx(tau, rel=1e-12)
        assert got[c]["sigma2"] == pytest.approx(1 / prec, rel=1e-12)
        assert np.array_equal(got[c]["x"], x0[c])


# --------------------------------------------------------------------------------------------
# Edge cases
# --------------------------------------------------------------------------------------------
EDGE = [
    ("1x1_2d4", lambda: wl.small_lattice(wl.LATTICE2D_4, (1, 1), 1)),
    ("1x1_2d8", lambda: wl.small_lattice(wl.LATTICE2D_8, (1, 1), 1)),
    ("1x1x1_3d6", lambda: wl.small_lattice(wl.LATTICE3D_6, (1, 1, 1), 1)),
    ("1x17_2d8", lambda: wl.small_lattice(wl.LATTICE2D_8, (1, 17), 2)),
    ("19x1_2d4", lambda: wl.small_lattice(wl.LATTICE2D_4, (19, 1), 3)),
    ("1x1x9_3d6", lambda: wl.small_lattice(wl.LATTICE3D_6, (1, 1, 9), 4)),
    ("csr_isolated", lambda: wl.graph_field(*wl.csr_from_edges(9, np.array([[0, 1], [2, 3], [3, 4]])), 5)),
    ("csr_star", lambda: wl.graph_field(*wl.star_graph(5000), 6)),
    ("csr_k40", lambda: wl.graph_field(*wl.random_graph(40, 1.01, wl.rng(1)), 7)),
    ("csr_single", lambda: wl.graph_field(np.array([0, 0]), np.zeros(0, np.int32), 8)),
]


@pytest.mark.parametrize("name,make", EDGE, ids=[e[0] for e in EDGE])
@pytest.mark.parametrize("precision", [g.FP32, g.FP64])
def test_edge_cases(name, make, precision):
    f = make()
    f["color_seed"] = 3
    T = 25
    res, _ = gpu_run([f], 3, T, precision, seed=67)
    compare(f, res[0], 3, T, 67, 0, 1e-4 if precision == g.FP32 else TOL_FP64)


def test_fixed_hyper_and_tau_zero():
    f = wl.small_lattice(wl.LATTICE2D_8, (20, 21), 9)
    res, _ = gpu_run([f], 2, 5, g.FP64, seed=71, fix_hyper=True, tau0=0.0, sigma2_0=0.49)
    st, out = compare(f, res[0], 2, 5, 71, 0, TOL_FP64, fix_hyper=True, tau0=0.0, sigma2_0=0.49)
    z = oracle.site_normals(71, f["n"], 4, 0, 1, oracle.lanes_for(2))
    np.testing.assert_allclose(res[0][1]["x"], f["y"] + 0.7 * z, rtol=1e-12, atol=1e-12)
    assert np.all(res[0][0]["tau_trace"] == 0.0)


def test_field_colours_reported():
    f = _delaunay(500, 17)
    lat = wl.small_lattice(wl.LATTICE2D_8, (6, 7), 1)
    with g.Sampler([f, lat], chains=1, seed=1) as s:
        c0, k0 = s.colors(0)
        c1, k1 = s.colors(1)
    want0 = oracle_colors(f)
    assert np.array_equal(c0, want0) and k0 == want0.max() + 1
    assert np.array_equal(c1, oracle.lattice_colors(oracle.LAT2D_8, (6, 7))[0]) and k1 == 4


# --------------------------------------------------------------------------------------------
# Fused one-launch-per-sweep 2-D lattice kernel vs the per-colour launches vs the oracle
# --------------------------------------------------------------------------------------------
FUSED = [("2d4_150x133", wl.LATTICE2D_4, (150, 133)), ("2d8_131x140", wl.LATTICE2D_8, (131, 140)),
         ("2d8_17x200", wl.LATTICE2D_8, (17, 200)), ("2d4_3x300", wl.LATTICE2D_4, (3, 300)),
         ("2d8_65x64", wl.LATTICE2D_8, (65, 64))]


@pytest.mark.parametrize("name,kind,dims", FUSED, ids=[c[0] for c in FUSED])
@pytest.mark.parametrize("chains", [1, 3, 8])
@pytest.mark.parametrize("flags", [0, g.FLAG_NO_RESIDENT, g.FLAG_PER_COLOUR], ids=["default", "fused", "per_colour"])
def test_lattice_paths_one_sweep(name, kind, dims, chains, flags):
    f = wl.small_lattice(kind, dims, 21)
    res, info = gpu_run([f], chains, 1, g.FP32, seed=73, flags=flags)
    compare(f, res[0], chains, 1, 73, 0, TOL_FP32_1)
    k = 4 if kind == wl.LATTICE2D_8 else 2
    assert info["launches_per_sweep"] == (k + 1 if flags == g.FLAG_PER_COLOUR else 2)


@pytest.mark.parametrize("precision,T,tol", [(g.FP32, 300, TOL_FP32_1000), (g.FP64, 100, TOL_FP64)])
@pytest.mark.parametrize("kind,dims", [(wl.LATTICE2D_8, (130, 97)), (wl.LATTICE2D_4, (99, 140))])
def test_fused_long_run(precision, T, tol, kind, dims):
    f = wl.small_lattice(kind, dims, 22)
    res, _ = gpu_run([f], 2, T, precision, seed=79, graph_sweeps=10, burn_in=T // 3)
    st, _ = compare(f, res[0], 2, T, 79, 0, tol, burn_in=T // 3)
    for c in range(2):
        assert relerr(res[0][c]["mean"], st.mean[c]) <= tol


def test_fused_and_per_colour_agree_to_rounding():
    f = wl.small_lattice(wl.LATTICE2D_8, (140, 150), 23)
    a, _ = gpu_run([f], 2, 50, g.FP64, seed=83)
    b, _ = gpu_run([f], 2, 50, g.FP64, seed=83, flags=g.FLAG_PER_COLOUR)
    for c in range(2):
        assert relerr(a[0][c]["x"], b[0][c]["x"]) <= TOL_FP64
        assert trace_relerr(a[0][c]["tau_trace"], b[0][c]["tau_trace"]) <= TOL_FP64


def test_stage_launch_diagnostic():
    fields = [wl.small_lattice(wl.LATTICE2D_8, (40, 40), 1), _delaunay(300, 2)]
    with g.Sampler(fields, chains=1, seed=3) as s:
        info = s.info()
        names = [s.launch_stage(k) for k in range(info["launches_per_sweep"])]
        with pytest.raises(g.GmrfError):
            s.launch_stage(info["launches_per_sweep"])
    assert names[0].startswith("fused") and "2-D 8-neighbour" in names[0]
    assert names[-1] == "hyperparameter draw"
    assert all(n.startswith("colour step, CSR") for n in names[1:-1])
