"""The oracle: a plain, slow FP64 CPU statement of the chromatic Gibbs sampler (Algorithm 1 of
Brown, McMahan & Self, arXiv 1702.05518) and of the generators it draws from.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (``paper_1702_05518_gb300``) never
imports it, and this package never imports the product: they share only the seeded input
generators of ``paper_1702_05518_gb300.workloads``, which hold none of the method's arithmetic.

The arithmetic lives in ``gmrf_oracle.c`` (plain C, FP64, single thread, built with
``-ffp-contract=off``); this module only marshals arguments through ctypes.

Parity status: every function here is pinned by ``tests/test_oracle_*.py`` against values the
paper or the mathematics fix (published Philox known answers, closed-form Gaussian conditionals
and posteriors, brute-force colourings, distribution tests).  The long-run posterior of tau and
sigma^2 is pinned only up to Monte Carlo error (compared with a dense block Gibbs sampler).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gmrf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libgmrf_oracle.so")
_lock = threading.Lock()
_lib = None

LAT2D_4, LAT2D_8, LAT3D_6 = 0, 1, 2
TAG_X, TAG_TAU, TAG_SIG, TAG_PRIO, TAG_BETA = 0, 1, 2, 3, 7


def build(force: bool = False) -> str:
    """Compile ``gmrf_oracle.c`` into ``oracle/_build/libgmrf_oracle.so`` (gcc, FP64, no FMA
    contraction so x86-64 and aarch64 give identical results)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _SO)
    return _SO


class _Model(ctypes.Structure):
    _fields_ = [("prior_proper", ctypes.c_int32), ("rho", ctypes.c_double),
                ("a_tau", ctypes.c_double), ("b_tau", ctypes.c_double),
                ("a_sig", ctypes.c_double), ("b_sig", ctypes.c_double),
                ("fix_hyper", ctypes.c_int32), ("intercept", ctypes.c_int32),
                ("binomial", ctypes.c_int32), ("beta0_mean", ctypes.c_double), ("beta0_var", ctypes.c_double)]


class _RunOpts(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("stream", ctypes.c_uint32),
                ("start_sweep", ctypes.c_uint32), ("nsweeps", ctypes.c_int32),
                ("burn_in", ctypes.c_int32), ("thin", ctypes.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            u32p, i32p, f64p, i64p = (P(ctypes.c_uint32), P(ctypes.c_int32),
                                      P(ctypes.c_double), P(ctypes.c_int64))
            lib.ora_philox4x32_10.argtypes = [u32p, u32p, u32p]
            lib.ora_philox_fill.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.c_uint32, ctypes.c_int64, u32p]
            lib.ora_uniform.argtypes = [ctypes.c_uint32]
            lib.ora_uniform.restype = ctypes.c_double
            lib.ora_normals4.argtypes = [u32p, f64p]
            lib.ora_lanes_for.argtypes = [ctypes.c_int32]
            lib.ora_lanes_for.restype = ctypes.c_int32
            lib.ora_site_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int32]
            lib.ora_site_normal.restype = ctypes.c_double
            lib.ora_site_normals.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_uint32,
                                             ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int32, f64p]
            lib.ora_gamma_draw.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                           ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                           ctypes.c_uint32, i32p]
            lib.ora_gamma_draw.restype = ctypes.c_double
            lib.ora_lattice_csr.argtypes = [ctypes.c_int32, i32p, i32p, i32p]
            lib.ora_lattice_csr.restype = ctypes.c_int64
            lib.ora_lattice_colors.argtypes = [ctypes.c_int32, i32p, i32p]
            lib.ora_lattice_colors.restype = ctypes.c_int32
            lib.ora_priorities.argtypes = [ctypes.c_uint64, ctypes.c_int32, u32p]
            lib.ora_priorities_ldf.argtypes = [ctypes.c_uint64, ctypes.c_int32, i32p, u32p]
            lib.ora_color_greedy.argtypes = [ctypes.c_int32, i32p, i32p, u32p, i32p]
            lib.ora_color_greedy.restype = ctypes.c_int32
            lib.ora_components.argtypes = [ctypes.c_int32, i32p, i32p]
            lib.ora_components.restype = ctypes.c_int32
            lib.ora_quadform.argtypes = [ctypes.c_int32, i32p, i32p, f64p, ctypes.c_double, f64p]
            lib.ora_quadform.restype = ctypes.c_double
            lib.ora_run.argtypes = [ctypes.c_int32, i32p, i32p, f64p, i32p, ctypes.c_int32, f64p, i32p,
                                    ctypes.c_int32, P(_Model), P(_RunOpts), f64p, f64p, f64p,
                                    f64p, f64p, f64p, f64p, f64p, f64p, i64p, f64p]
            lib.ora_run.restype = ctypes.c_int32
            lib.ora_beta_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.c_uint32, ctypes.c_uint32]
            lib.ora_beta_normal.restype = ctypes.c_double
            lib.ora_pg_draw.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                                        ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, P(ctypes.c_int32)]
            lib.ora_pg_draw.restype = ctypes.c_double
            lib.ora_pg_term.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_int32]
            lib.ora_pg_term.restype = ctypes.c_double
            lib.ora_pg_mix_weight.argtypes = [ctypes.c_double]
            lib.ora_pg_mix_weight.restype = ctypes.c_double
            lib.ora_iat.argtypes = [f64p, ctypes.c_int64]
            lib.ora_iat.restype = ctypes.c_double
            lib.ora_psrf.argtypes = [f64p, ctypes.c_int32, ctypes.c_int64]
            lib.ora_psrf.restype = ctypes.c_double
            lib.ora_psrf_moments.argtypes = [f64p, f64p, ctypes.c_int32, ctypes.c_int64]
            lib.ora_psrf_moments.restype = ctypes.c_double
            _lib = lib
    return _lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------------------------
# Generators
# --------------------------------------------------------------------------------------------
def philox(ctr, key):
    """Philox4x32-10 of one 4-word counter under a 2-word key -> 4 uint32 words."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib.ora_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                          _ptr(out, ctypes.c_uint32))
    return out


def philox_fill(seed, c1, c2, c3, n):
    """Philox blocks for counters (i, c1, c2, c3), i = 0..n-1, key = (seed lo, seed hi): [n, 4]."""
    out = np.zeros((int(n), 4), np.uint32)
    _load().ora_philox_fill(seed, c1, c2, c3, int(n), _ptr(out, ctypes.c_uint32))
    return out


def uniform(w):
    return _load().ora_uniform(int(w))


def normals4(words):
    w = np.ascontiguousarray(words, dtype=np.uint32)
    z = np.zeros(4, np.float64)
    _load().ora_normals4(_ptr(w, ctypes.c_uint32), _ptr(z, ctypes.c_double))
    return z


def lanes_for(chains):
    """Normals per site of one Philox block for a sampler with `chains` chains: 1, 2 or 4."""
    return _load().ora_lanes_for(int(chains))


def site_normal(seed, site, sweep, stream, chain, lanes):
    return _load().ora_site_normal(seed, site, sweep, stream, chain, lanes)


def site_normals(seed, n, sweep, stream, chain, lanes):
    """Normals z_i used to update sites 0..n-1 of `chain` at `sweep` (natural site order) in a
    sampler whose Philox blocks serve `lanes` chains (see lanes_for)."""
    out = np.zeros(int(n), np.float64)
    _load().ora_site_normals(seed, int(n), sweep, stream, chain, int(lanes), _ptr(out, ctypes.c_double))
    return out


def gamma_draw(shape, rate, seed, sweep, stream, tag, chain):
    """Gamma(shape, rate) by Marsaglia-Tsang with the Philox counters of the hyper draws.
    Returns (value, attempts); attempts is -1 when the 64-attempt limit was hit."""
    att = ctypes.c_int32(0)
    g = _load().ora_gamma_draw(float(shape), float(rate), seed, sweep, stream, tag, chain,
                               ctypes.byref(att))
    return g, att.value


def pg_draw(b, c, seed, site=0, sweep=0, stream=0, chain=0):
    """A Polya-Gamma PG(b, c) variate (sum of b PG(1, c) by Devroye's method) with the counters of
    the draw of (site, sweep, chain).  Returns (value, fallbacks)."""
    fb = ctypes.c_int32(0)
    v = _load().ora_pg_draw(int(b), float(c), seed, site, sweep, stream, chain, ctypes.byref(fb))
    return v, fb.value


def pg_series_term(n, x, form):
    """Term n of the alternating series of the J*(1, 0) density: small-x form (0) or large-x (1)."""
    return _load().ora_pg_term(int(n), float(x), int(form))


def pg_mix_weight(z):
    """Probability of the exponential piece of the J*(1, z) proposal."""
    return _load().ora_pg_mix_weight(float(z))


def beta_normal(seed, sweep, stream, chain, tag=TAG_BETA):
    """Standard normal of the intercept draw: Box-Muller cosine of words (w0, w1) of the Philox
    block at counter (0, sweep, stream, (tag << 24) | chain)."""
    return _load().ora_beta_normal(seed, sweep, stream, tag, chain)


# --------------------------------------------------------------------------------------------
# Graphs and colourings
# --------------------------------------------------------------------------------------------
def _dims3(dims):
    d = list(dims) + [0] * (3 - len(dims))
    return np.ascontiguousarray(d[:3], dtype=np.int32)


def lattice_n(kind, dims):
    return int(np.prod(dims[:3] if kind == LAT3D_6 else dims[:2]))


def lattice_csr(kind, dims):
    """CSR (row_ptr, col_idx) of a free-boundary lattice in row-major site order."""
    lib = _load()
    d = _dims3(dims)
    n = lattice_n(kind, dims)
    nnz = lib.ora_lattice_csr(kind, _ptr(d, ctypes.c_int32), None, None)
    rp = np.zeros(n + 1, np.int32)
    ci = np.zeros(max(nnz, 1), np.int32)
    lib.ora_lattice_csr(kind, _ptr(d, ctypes.c_int32), _ptr(rp, ctypes.c_int32),
                        _ptr(ci, ctypes.c_int32))
    return rp, ci[:nnz]


def lattice_colors(kind, dims):
    d = _dims3(dims)
    colors = np.zeros(lattice_n(kind, dims), np.int32)
    k = _load().ora_lattice_colors(kind, _ptr(d, ctypes.c_int32), _ptr(colors, ctypes.c_int32))
    return colors, k


def priorities(seed, n):
    p = np.zeros(int(n), np.uint32)
    _load().ora_priorities(seed, int(n), _ptr(p, ctypes.c_uint32))
    return p


def priorities_ldf(seed, row_ptr):
    """Largest-degree-first priorities: min(degree, 255) in the top 8 bits, the top 24 bits of the
    random priority of `seed` below."""
    rp = _i32(row_ptr)
    n = len(rp) - 1
    p = np.zeros(n, np.uint32)
    _load().ora_priorities_ldf(seed, int(n), _ptr(rp, ctypes.c_int32), _ptr(p, ctypes.c_uint32))
    return p


def color_greedy(row_ptr, col_idx, prio):
    """First-fit greedy colouring in decreasing (priority, index) order -> (colors, k)."""
    rp, ci = _i32(row_ptr), _i32(col_idx)
    n = len(rp) - 1
    pr = np.ascontiguousarray(prio, dtype=np.uint32)
    colors = np.zeros(n, np.int32)
    k = _load().ora_color_greedy(n, _ptr(rp, ctypes.c_int32), _ptr(ci, ctypes.c_int32),
                                 _ptr(pr, ctypes.c_uint32), _ptr(colors, ctypes.c_int32))
    return colors, k


def color_graph(row_ptr, col_idx, seed, ldf=False):
    """The colouring a graph gets from its seed: greedy in decreasing Philox-priority order
    (largest degree first with ldf)."""
    n = len(row_ptr) - 1
    prio = priorities_ldf(seed, row_ptr) if ldf else priorities(seed, n)
    return color_greedy(row_ptr, col_idx, prio)


def components(row_ptr, col_idx):
    rp, ci = _i32(row_ptr), _i32(col_idx)
    return _load().ora_components(len(rp) - 1, _ptr(rp, ctypes.c_int32), _ptr(ci, ctypes.c_int32))


def quadform(row_ptr, col_idx, x, rho=1.0, weights=None):
    rp, ci, xx = _i32(row_ptr), _i32(col_idx), _f64(x)
    w = None if weights is None else _f64(weights)
    return _load().ora_quadform(len(rp) - 1, _ptr(rp, ctypes.c_int32), _ptr(ci, ctypes.c_int32),
                                _ptr(w, ctypes.c_double), float(rho), _ptr(xx, ctypes.c_double))


# --------------------------------------------------------------------------------------------
# The sampler
# --------------------------------------------------------------------------------------------
class State:
    """Chain state of one field: x [C, n], tau [C], sigma2 [C], the intercept beta0 [C] and the
    Welford accumulators."""

    def __init__(self, x, tau, sigma2, mean=None, m2=None, count=0, beta0=None):
        self.x = np.array(x, dtype=np.float64, order="C")
        C, n = self.x.shape
        self.tau = np.array(tau, dtype=np.float64).reshape(C).copy()
        self.sigma2 = np.array(sigma2, dtype=np.float64).reshape(C).copy()
        self.beta0 = np.zeros(C) if beta0 is None else np.array(beta0, dtype=np.float64).reshape(C).copy()
        self.mean = np.zeros((C, n)) if mean is None else np.array(mean, dtype=np.float64)
        self.m2 = np.zeros((C, n)) if m2 is None else np.array(m2, dtype=np.float64)
        self.count = int(count)

    def copy(self):
        return State(self.x, self.tau, self.sigma2, self.mean, self.m2, self.count, self.beta0)


def run(graph, colors, y, state, *, seed, nsweeps, stream=0, start_sweep=0, prior="icar",
        rho=1.0, a_tau=1.0, b_tau=0.01, a_sig=1.0, b_sig=0.01, fix_hyper=False, burn_in=0,
        thin=1, accumulate=True, record_x=False, weights=None, intercept=False, trials=None,
        beta0_prior=(0.0, 1000.0)):
    """Run `nsweeps` chromatic Gibbs sweeps (Algorithm 1 + conjugate tau, sigma^2 draws, and with
    `intercept` the flat-prior beta0 draw of Sec. 3.1) of every chain in `state` (modified in
    place).  graph = (row_ptr, col_idx) in natural order.  With `trials` (m_i per site) the data
    are binomial, y_i ~ Bin(m_i, logistic(beta0 + x_i)) (Sec. 3.2): Polya-Gamma augmentation,
    beta0 ~ N(beta0_prior), no sigma^2.

    Returns dict(tau_trace [C, T], sigma2_trace [C, T], beta0_trace [C, T], fallbacks,
    xtrace [T, C, n] or None).
    """
    lib = _load()
    rp, ci = _i32(graph[0]), _i32(graph[1])
    n = len(rp) - 1
    col = _i32(colors)
    k = int(col.max()) + 1 if n > 0 else 0
    yy = _f64(y)
    C = state.x.shape[0]
    assert state.x.shape == (C, n) and yy.shape == (n,)
    w = None if weights is None else _f64(weights)
    model = _Model(1 if prior == "pcar" else 0, float(rho), float(a_tau), float(b_tau),
                   float(a_sig), float(b_sig), 1 if fix_hyper else 0, 1 if intercept else 0,
                   0 if trials is None else 1, float(beta0_prior[0]), float(beta0_prior[1]))
    tr = None if trials is None else _i32(trials)
    opts = _RunOpts(int(seed), int(stream), int(start_sweep), int(nsweeps), int(burn_in),
                    int(thin))
    tt = np.zeros((C, max(nsweeps, 1)))
    st = np.zeros((C, max(nsweeps, 1)))
    bt = np.zeros((C, max(nsweeps, 1)))
    xt = np.zeros((max(nsweeps, 1), C, n)) if record_x else None
    cnt = ctypes.c_int64(state.count)
    fb = lib.ora_run(n, _ptr(rp, ctypes.c_int32), _ptr(ci, ctypes.c_int32),
                     _ptr(w, ctypes.c_double), _ptr(col, ctypes.c_int32), k,
                     _ptr(yy, ctypes.c_double), _ptr(tr, ctypes.c_int32), C, ctypes.byref(model),
                     ctypes.byref(opts),
                     _ptr(state.x, ctypes.c_double), _ptr(state.tau, ctypes.c_double),
                     _ptr(state.sigma2, ctypes.c_double), _ptr(state.beta0, ctypes.c_double),
                     _ptr(tt, ctypes.c_double), _ptr(st, ctypes.c_double), _ptr(bt, ctypes.c_double),
                     _ptr(state.mean, ctypes.c_double) if accumulate else None,
                     _ptr(state.m2, ctypes.c_double) if accumulate else None,
                     ctypes.byref(cnt) if accumulate else None,
                     _ptr(xt, ctypes.c_double))
    if accumulate:
        state.count = cnt.value
    return {"tau_trace": tt[:, :nsweeps], "sigma2_trace": st[:, :nsweeps],
            "beta0_trace": bt[:, :nsweeps], "fallbacks": fb,
            "xtrace": xt[:nsweeps] if record_x else None}


def initial_state(y, chains, tau0=1.0, sigma2_0=1.0, x0=None, beta0=0.0):
    """x0 = y for every chain unless given ([C, n] or [n]); tau0, sigma2_0, beta0 scalars or [C]."""
    y = _f64(y)
    if x0 is None:
        x = np.tile(y, (chains, 1))
    else:
        x0 = np.asarray(x0, dtype=np.float64)
        x = np.tile(x0, (chains, 1)) if x0.ndim == 1 else x0.copy()
    tau = np.broadcast_to(np.asarray(tau0, dtype=np.float64), (chains,)).copy()
    sig = np.broadcast_to(np.asarray(sigma2_0, dtype=np.float64), (chains,)).copy()
    b0 = np.broadcast_to(np.asarray(beta0, dtype=np.float64), (chains,)).copy()
    return State(x, tau, sig, beta0=b0)


# --------------------------------------------------------------------------------------------
# Chain diagnostics
# --------------------------------------------------------------------------------------------
def iat(x):
    """Integrated autocorrelation time by Geyer's initial monotone sequence (NaN if undefined)."""
    xx = _f64(x)
    return _load().ora_iat(_ptr(xx, ctypes.c_double), len(xx))


def ess(x):
    """Effective sample size N / IAT."""
    return len(x) / iat(x)


def psrf(chains):
    """Potential scale reduction factor of chains [m, N] (Brooks-Gelman form)."""
    xx = np.ascontiguousarray(chains, dtype=np.float64)
    m, N = xx.shape
    return _load().ora_psrf(_ptr(xx, ctypes.c_double), m, N)


def psrf_moments(means, variances, N):
    """PSRF from per-chain means and variances (divisor N - 1) of N values each."""
    mu, var = _f64(means), _f64(variances)
    return _load().ora_psrf_moments(_ptr(mu, ctypes.c_double), _ptr(var, ctypes.c_double), len(mu), int(N))

