"""Long coupled runs at the benchmark's kernels and launch configuration, compared with the
oracle element by element (FP32 bar after 1000 coupled sweeps: 1e-4 on x, on the posterior mean
and on the tau and sigma^2 traces, relative to max(|oracle|, 1)).

- the quad kernel (single-chain FP32 8-neighbour lattice) at the full 1024 x 1024 size of the
  default image workload: 1000 sweeps, the last 500 accumulated, CUDA graphs of 50 sweeps;
- the 3-D colour step with every chain of a site in one thread, on a 48^3 ellipsoid volume
  (one wave of tiles with ragged row ranges) with 8 chains: 1000 sweeps, the last 500
  accumulated, CUDA graphs of 25 sweeps.

The oracle runs take a minute or two each on one core; they start in background threads when
the module is collected (the oracle is C called through ctypes, which releases the GIL) and the
GPU runs proceed meanwhile.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from gmrf_testutil import TOL_FP32_1000, relerr, run_oracle, trace_relerr
from paper_1702_05518_gb300 import gmrf as g
from paper_1702_05518_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

T, BURN = 1000, 500


def _image():
    return wl.image_1024_bumps(seed=2)[0], 1, 2, 50


def _volume():
    return wl.volume_ellipsoids(seed=5, side=48)[0], 8, 5, 25


CASES = {"image1024_quad": _image, "volume48_c8": _volume}


@pytest.fixture(scope="module")
def oracle_runs():
    pool = ThreadPoolExecutor(max_workers=len(CASES))
    futs = {}
    for name, make in CASES.items():
        f, C, seed, _ = make()
        futs[name] = pool.submit(run_oracle, f, C, T, seed=seed, stream=0, burn_in=BURN)
    yield futs
    pool.shutdown(wait=True)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1702_05518_gb300 import build

    build.build()


@pytest.mark.parametrize("name", list(CASES))
def test_1000_coupled_sweeps(name, oracle_runs):
    f, C, seed, G = CASES[name]()
    with g.Sampler([f], precision=g.FP32, chains=C, seed=seed, burn_in=BURN, graph_sweeps=G) as s:
        s.sweep(T)
        res = [s.fetch(0, c, trace=T) for c in range(C)]
        info = s.info()
    st, out = oracle_runs[name].result()
    worst = {"x": 0.0, "mean": 0.0, "tau": 0.0, "sigma2": 0.0}
    for c in range(C):
        worst["x"] = max(worst["x"], relerr(res[c]["x"], st.x[c]))
        worst["mean"] = max(worst["mean"], relerr(res[c]["mean"], st.mean[c]))
        worst["tau"] = max(worst["tau"], trace_relerr(res[c]["tau_trace"], out["tau_trace"][c]))
        worst["sigma2"] = max(worst["sigma2"], trace_relerr(res[c]["sigma2_trace"], out["sigma2_trace"][c]))
    assert max(worst.values()) <= TOL_FP32_1000, worst
    assert info["accumulated"] == T - BURN and info["hyper_fallbacks"] == 0
