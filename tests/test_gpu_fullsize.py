"""GPU parity at the full sizes of the benchmark workloads, in the launch configuration the
benchmark times (CUDA graphs of several sweeps), compared with the oracle element by element.

- 1024 x 1024 8-neighbour ICAR, 2x2 colouring, 20 Gaussian bumps + N(0,1), FP32, 1 chain.
- 256^3 6-neighbour ICAR, parity colouring, 50 ellipsoids + N(0,1), FP32, 8 chains.
- Delaunay graph of 16384 points, proper CAR rho = 0.95, prior-drawn truth, FP32, 8 chains (coloured
  with random priorities, and largest degree first).
- 224 lattices + 32 Delaunay graphs of uneven sizes in one batched sampler, FP32.
"""
import numpy as np
import pytest

from gmrf_testutil import TOL_FP32_1, TOL_FP32_1000, relerr, run_oracle, trace_relerr
from paper_1702_05518_gb300 import gmrf as g
from paper_1702_05518_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

BENCH_GRAPH_SWEEPS = 20


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1702_05518_gb300 import build

    build.build()


def _check(fields, chains, nsweeps, seed, tol, **kw):
    okw = {k: v for k, v in kw.items() if k in ("rho",)}
    if kw.get("prior") == g.PRIOR_PCAR:
        okw["prior"] = "pcar"
    with g.Sampler(fields, precision=g.FP32, chains=chains, seed=seed,
                   graph_sweeps=BENCH_GRAPH_SWEEPS, **kw) as s:
        s.sweep(nsweeps)
        got = [[s.fetch(f, c, trace=nsweeps) for c in range(chains)] for f in range(len(fields))]
    worst = 0.0
    for fi, f in enumerate(fields):
        st, out = run_oracle(f, chains, nsweeps, seed=seed, stream=fi, **okw)
        for c in range(chains):
            worst = max(worst, relerr(got[fi][c]["x"], st.x[c]),
                        trace_relerr(got[fi][c]["tau_trace"], out["tau_trace"][c]),
                        trace_relerr(got[fi][c]["sigma2_trace"], out["sigma2_trace"][c]))
    assert worst <= tol, f"{worst:.3e} > {tol:.1e}"


def test_image_1024_bumps_full_size():
    f = wl.image_1024_bumps(seed=2)
    _check(f, 1, 1, 2, TOL_FP32_1)
    _check(f, 1, 25, 2, TOL_FP32_1000)


def test_volume_256_ellipsoids_full_size():
    f = wl.volume_ellipsoids(seed=5)
    _check(f, 8, 1, 5, TOL_FP32_1)


@pytest.mark.parametrize("random", [True, False], ids=["random_priorities", "largest_degree_first"])
def test_delaunay_16k_pcar_full_size(random):
    # the workload's colouring (Jones-Plassmann, random 32-bit priorities) and the sampler's default
    f = wl.delaunay_pcar(seed=3)
    f[0]["color_seed"] = 3
    f[0]["color_random"] = random
    flags = g.FLAG_COLOR_RANDOM if random else 0
    _check(f, 8, 1, 3, TOL_FP32_1, prior=g.PRIOR_PCAR, rho=0.95, flags=flags)
    _check(f, 8, 200, 3, TOL_FP32_1000, prior=g.PRIOR_PCAR, rho=0.95, flags=flags)


def test_batched_uneven_full_size():
    fields = wl.batched_uneven(seed=4)
    for i, f in enumerate(fields):
        f["color_seed"] = 100 + i
    _check(fields, 1, 1, 4, TOL_FP32_1)
