"""Helpers shared by the GPU parity tests: run the oracle on the same seeded inputs a sampler
got, and compare with the parity metric |x_gpu - x_oracle| / max(|x_oracle|, 1)."""
import numpy as np

import oracle
from paper_1702_05518_gb300 import workloads as wl

KIND_TO_ORACLE = {wl.LATTICE2D_4: oracle.LAT2D_4, wl.LATTICE2D_8: oracle.LAT2D_8,
                  wl.LATTICE3D_6: oracle.LAT3D_6}

# Parity tolerances (max relative error with denominator max(|x|, 1)): FP32 state after one
# sweep / after 1000 coupled sweeps, and FP64.
TOL_FP32_1 = 1e-5
TOL_FP32_1000 = 1e-4
TOL_FP64 = 1e-12


def oracle_graph(field):
    if field["kind"] == wl.CSR:
        return field["row_ptr"], field["col_idx"]
    return oracle.lattice_csr(KIND_TO_ORACLE[field["kind"]], field["dims"])


def oracle_colors(field):
    if field["kind"] == wl.CSR:
        if field.get("colors") is not None:
            return np.asarray(field["colors"], np.int32)
        # the sampler's own colouring: largest degree first unless the field asks for random
        # priorities (sampled with GMRF_FLAG_COLOR_RANDOM)
        return oracle.color_graph(field["row_ptr"], field["col_idx"], field.get("color_seed", 0),
                                  ldf=not field.get("color_random", False))[0]
    return oracle.lattice_colors(KIND_TO_ORACLE[field["kind"]], field["dims"])[0]


def run_oracle(field, chains, nsweeps, *, seed, stream, prior="icar", rho=1.0, start_sweep=0,
               fix_hyper=False, burn_in=0, thin=1, tau0=1.0, sigma2_0=1.0, a_tau=1.0, b_tau=0.01,
               a_sig=1.0, b_sig=0.01, record_x=False, intercept=False, beta0=0.0):
    st = oracle.initial_state(field["y"], chains, tau0=field.get("tau0", tau0),
                              sigma2_0=field.get("sigma2_0", sigma2_0), x0=field.get("x0"),
                              beta0=field.get("beta0", beta0))
    out = oracle.run(oracle_graph(field), oracle_colors(field), field["y"], st, seed=seed,
                     nsweeps=nsweeps, stream=stream, start_sweep=start_sweep, prior=prior, rho=rho,
                     fix_hyper=fix_hyper, burn_in=burn_in, thin=thin, a_tau=a_tau, b_tau=b_tau,
                     a_sig=a_sig, b_sig=b_sig, weights=field.get("weights"), record_x=record_x,
                     intercept=intercept)
    return st, out


def relerr(got, want):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    if got.size == 0:
        return 0.0
    return float(np.max(np.abs(got - want) / np.maximum(np.abs(want), 1.0)))


def trace_relerr(got, want):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    if got.size == 0:
        return 0.0
    # relative to the value; absolute where the value is 0 (a trace of tau fixed at 0)
    diff = np.abs(got - want)
    den = np.abs(want)
    return float(np.max(np.where(den > 0, diff / np.where(den > 0, den, 1.0), diff)))
