"""Thin ctypes binding of libgmrf (include/gmrf.h): argument marshalling only.

Every step of the sampler runs in the CUDA library; this module converts numpy inputs to the C
structs, passes PyTorch's current CUDA stream, and copies results back into numpy arrays.  If
the library has not been built, loading fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgmrf.so")

OK, E_INVALID, E_CUDA, E_OOM, E_STATE, E_TIMEOUT, E_UNSUPPORTED = range(7)
LATTICE2D_4, LATTICE2D_8, LATTICE3D_6, CSR = range(4)
PRIOR_ICAR, PRIOR_PCAR = 0, 1
FP32, FP64 = 0, 1
ALGO_CHROMATIC, ALGO_PLAIN = 0, 1
FLAG_PER_COLOUR = 1
FLAG_NO_RESIDENT = 2
FLAG_RESIDENT = 4
FLAG_TEST_STALL = 8
FLAG_COLOR_RANDOM = 16
PARAM_TAU2, PARAM_SIGMA2, PARAM_BETA0, PARAM_TAU = range(4)
LIKELIHOOD_GAUSSIAN, LIKELIHOOD_BINOMIAL = 0, 1

EXPORTED = ["gmrf_color_graph", "gmrf_color_graph_noalloc", "gmrf_sampler_create", "gmrf_sampler_destroy", "gmrf_sweep",
            "gmrf_hyper_update", "gmrf_fetch_samples", "gmrf_field_colors", "gmrf_sampler_info",
            "gmrf_sampler_reset", "gmrf_sampler_set_data", "gmrf_launch_stage", "gmrf_fetch_intercept",
            "gmrf_trace_diagnostics", "gmrf_site_psrf", "gmrf_autotune",
            "gmrf_validate_csr", "gmrf_philox_words", "gmrf_site_normals", "gmrf_normals_timing", "gmrf_fetch_pooled",
            "gmrf_debug_fail_alloc",
            "gmrf_debug_poison", "gmrf_last_error", "gmrf_version"]


class GmrfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"gmrf status {status}: {msg}")
        self.status = status


class FieldDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dims", ctypes.c_int32 * 3), ("n", ctypes.c_int32),
                ("row_ptr", ctypes.POINTER(ctypes.c_int32)),
                ("col_idx", ctypes.POINTER(ctypes.c_int32)),
                ("weights", ctypes.POINTER(ctypes.c_double)),
                ("colors", ctypes.POINTER(ctypes.c_int32)), ("color_seed", ctypes.c_uint64),
                ("y", ctypes.POINTER(ctypes.c_double)), ("x0", ctypes.POINTER(ctypes.c_double)),
                ("tau0", ctypes.POINTER(ctypes.c_double)),
                ("sigma2_0", ctypes.POINTER(ctypes.c_double)), ("stream_id", ctypes.c_uint32),
                ("beta0", ctypes.POINTER(ctypes.c_double)),
                ("trials", ctypes.POINTER(ctypes.c_int32))]


class Model(ctypes.Structure):
    _fields_ = [("prior", ctypes.c_int32), ("rho", ctypes.c_double), ("a_tau", ctypes.c_double),
                ("b_tau", ctypes.c_double), ("a_sigma", ctypes.c_double),
                ("b_sigma", ctypes.c_double), ("fix_hyper", ctypes.c_int32),
                ("tau0", ctypes.c_double), ("sigma2_0", ctypes.c_double),
                ("intercept", ctypes.c_int32), ("beta0_0", ctypes.c_double),
                ("likelihood", ctypes.c_int32), ("beta0_mean", ctypes.c_double), ("beta0_var", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("chains_per_thread", ctypes.c_int32), ("step_tile", ctypes.c_int32),
                ("fused_rows", ctypes.c_int32 * 2), ("fused_cols", ctypes.c_int32 * 2),
                ("fused_threads", ctypes.c_int32 * 2), ("quad_config", ctypes.c_int32),
                ("quad_rows", ctypes.c_int32), ("wide_3d", ctypes.c_int32), ("graph_cluster", ctypes.c_int32)]

    @classmethod
    def from_dict(cls, d):
        t = cls()
        for k, v in (d or {}).items():
            if k in ("fused_rows", "fused_cols", "fused_threads"):
                arr = getattr(t, k)
                for i, x in enumerate(v):
                    arr[i] = int(x)
            else:
                setattr(t, k, int(v))
        return t

    def to_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if k.startswith("fused_") else int(v)
        return out


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("chains", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("start_sweep", ctypes.c_int64),
                ("burn_in", ctypes.c_int64), ("thin", ctypes.c_int32),
                ("trace_capacity", ctypes.c_int32), ("algorithm", ctypes.c_int32),
                ("graph_sweeps", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("tuning", ctypes.POINTER(Tuning))]


class Info(ctypes.Structure):
    _fields_ = [("nfields", ctypes.c_int32), ("chains", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("max_colors", ctypes.c_int32),
                ("sweeps_done", ctypes.c_int64), ("accumulated", ctypes.c_int64),
                ("hyper_fallbacks", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("launches_per_sweep", ctypes.c_int64), ("early_start_misses", ctypes.c_int64),
                ("resident", ctypes.c_int64), ("wait_timeouts", ctypes.c_int64)]


_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """Load libgmrf.so (raises if it is missing: build it with ``__graft_entry__.build()``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: the CUDA library must be built "
                                  "(python -c 'import __graft_entry__ as g; g.build()')")
            L = ctypes.CDLL(LIB_PATH)
            P = ctypes.POINTER
            i32p, u32p, f64p, i64p = (P(ctypes.c_int32), P(ctypes.c_uint32), P(ctypes.c_double),
                                      P(ctypes.c_int64))
            st = ctypes.c_int
            vp = ctypes.c_void_p
            L.gmrf_color_graph.argtypes = [ctypes.c_int32, i32p, i32p, u32p, ctypes.c_uint64, i32p, i32p]
            L.gmrf_color_graph.restype = st
            L.gmrf_color_graph_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int64, vp, vp, vp, ctypes.c_uint64,
                                                   vp, i32p, vp]
            L.gmrf_color_graph_noalloc.restype = st
            L.gmrf_sampler_create.argtypes = [P(vp), P(FieldDesc), ctypes.c_int32, P(Model), P(Opts), vp]
            L.gmrf_sampler_create.restype = st
            L.gmrf_sampler_destroy.argtypes = [vp]
            L.gmrf_sampler_destroy.restype = None
            L.gmrf_sweep.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
            L.gmrf_sweep.restype = st
            L.gmrf_sampler_reset.argtypes = [vp]
            L.gmrf_sampler_reset.restype = st
            L.gmrf_sampler_set_data.argtypes = [vp, ctypes.c_int32, f64p, i32p, f64p]
            L.gmrf_sampler_set_data.restype = st
            L.gmrf_autotune.argtypes = [P(FieldDesc), ctypes.c_int32, P(Model), P(Opts), ctypes.c_int32, vp,
                                        P(Tuning), f64p]
            L.gmrf_autotune.restype = st
            L.gmrf_launch_stage.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, P(ctypes.c_char_p)]
            L.gmrf_launch_stage.restype = st
            L.gmrf_hyper_update.argtypes = [vp]
            L.gmrf_hyper_update.restype = st
            L.gmrf_fetch_samples.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, f64p, f64p, f64p,
                                             ctypes.c_int64, f64p, f64p, i64p, f64p, f64p]
            L.gmrf_fetch_samples.restype = st
            L.gmrf_fetch_intercept.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, f64p, i64p,
                                               f64p]
            L.gmrf_fetch_intercept.restype = st
            L.gmrf_trace_diagnostics.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, f64p, f64p,
                                                 f64p]
            L.gmrf_trace_diagnostics.restype = st
            L.gmrf_site_psrf.argtypes = [vp, ctypes.c_int32, f64p, f64p]
            L.gmrf_site_psrf.restype = st
            L.gmrf_field_colors.argtypes = [vp, ctypes.c_int32, i32p, i32p]
            L.gmrf_field_colors.restype = st
            L.gmrf_sampler_info.argtypes = [vp, P(Info)]
            L.gmrf_sampler_info.restype = st
            L.gmrf_validate_csr.argtypes = [ctypes.c_int32, i32p, i32p, f64p, i32p]
            L.gmrf_validate_csr.restype = st
            L.gmrf_philox_words.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.c_uint32, ctypes.c_int64, vp, vp]
            L.gmrf_philox_words.restype = st
            L.gmrf_site_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.c_uint32, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int64, vp, vp]
            L.gmrf_site_normals.restype = st
            L.gmrf_normals_timing.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, vp,
                                              f64p]
            L.gmrf_normals_timing.restype = st
            L.gmrf_fetch_pooled.argtypes = [vp, ctypes.c_int32, f64p, f64p]
            L.gmrf_fetch_pooled.restype = st
            L.gmrf_debug_fail_alloc.argtypes = [ctypes.c_int64]
            L.gmrf_debug_fail_alloc.restype = st
            L.gmrf_debug_poison.argtypes = [vp]
            L.gmrf_debug_poison.restype = st
            L.gmrf_last_error.argtypes = []
            L.gmrf_last_error.restype = ctypes.c_char_p
            L.gmrf_version.argtypes = []
            L.gmrf_version.restype = ctypes.c_char_p
            _lib = L
    return _lib


def _check(status):
    if status != OK:
        raise GmrfError(status, lib().gmrf_last_error().decode())


def _p(a, ct):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ct))


def _i32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def current_stream():
    """PyTorch's current CUDA stream handle (or None: the legacy default stream)."""
    try:
        import torch

        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


def validate_csr(row_ptr, col_idx, weights=None):
    """Host-only CSR check; returns the number of connected components."""
    rp, ci, w = _i32(row_ptr), _i32(col_idx), _f64(weights)
    comps = ctypes.c_int32(0)
    _check(lib().gmrf_validate_csr(len(rp) - 1, _p(rp, ctypes.c_int32), _p(ci, ctypes.c_int32),
                                   _p(w, ctypes.c_double), ctypes.byref(comps)))
    return comps.value


def color_graph(row_ptr, col_idx, seed=0, priorities=None):
    """Jones-Plassmann colouring on the GPU -> (colors [n] int32, k)."""
    rp, ci = _i32(row_ptr), _i32(col_idx)
    n = len(rp) - 1
    pr = None if priorities is None else np.ascontiguousarray(priorities, dtype=np.uint32)
    colors = np.zeros(n, np.int32)
    k = ctypes.c_int32(0)
    _check(lib().gmrf_color_graph(n, _p(rp, ctypes.c_int32), _p(ci, ctypes.c_int32),
                                  _p(pr, ctypes.c_uint32), int(seed), _p(colors, ctypes.c_int32),
                                  ctypes.byref(k)))
    return colors, k.value


def color_graph_noalloc(row_ptr, col_idx, colors, priorities=None, seed=0):
    """gmrf_color_graph_noalloc on device tensors (int32 row_ptr [n+1], col_idx [nnz], colors
    [n] out; optional int32/uint32 priorities [n]) on the current stream -> number of colours.
    Raises ValueError, before any call, unless every tensor is contiguous, of those types and
    sizes, and on the current CUDA device (the library reads and writes them as device arrays)."""
    import torch

    n = int(row_ptr.numel()) - 1
    named = [("row_ptr", row_ptr, (torch.int32,), None), ("col_idx", col_idx, (torch.int32,), None),
             ("colors", colors, (torch.int32,), n)]
    if priorities is not None:
        named.append(("priorities", priorities, (torch.int32, torch.uint32), n))
    for name, t, dtypes, size in named:
        if t.dtype not in dtypes:
            raise ValueError(f"{name} must be {' or '.join(str(d) for d in dtypes)}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if size is not None and int(t.numel()) != size:
            raise ValueError(f"{name} has {t.numel()} elements, expected n = {size}")
    if n < 0:
        raise ValueError("row_ptr must have n + 1 >= 1 elements")
    dev = torch.cuda.current_device() if torch.cuda.is_available() else None
    for name, t, _, _ in named:
        if not t.is_cuda or t.device.index != dev:
            raise ValueError(f"{name} must be on the current CUDA device")
    k = ctypes.c_int32(0)
    pr = None if priorities is None else ctypes.c_void_p(priorities.data_ptr())
    _check(lib().gmrf_color_graph_noalloc(n, int(col_idx.numel()), ctypes.c_void_p(row_ptr.data_ptr()),
                                          ctypes.c_void_p(col_idx.data_ptr()), pr, int(seed),
                                          ctypes.c_void_p(colors.data_ptr()), ctypes.byref(k),
                                          current_stream()))
    return k.value


def normals_timing(seed, sites, chains, reps=20):
    """Microseconds per launch of the 3-D colour step's normals alone (sites x chains normals)."""
    us = ctypes.c_double(0)
    _check(lib().gmrf_normals_timing(int(seed), int(sites), int(chains), int(reps), current_stream(), ctypes.byref(us)))
    return us.value


def debug_fail_alloc(nth):
    """Make the nth device allocation of the library from now on fail as out of memory (0: off)."""
    _check(lib().gmrf_debug_fail_alloc(int(nth)))


def philox_words(seed, c1, c2, c3, count):
    """Philox4x32-10 words of counters (i, c1, c2, c3), i < count, computed on the GPU: [count, 4]."""
    import torch

    out = torch.empty(int(count) * 4, dtype=torch.int32, device="cuda")
    _check(lib().gmrf_philox_words(int(seed), c1, c2, c3, int(count), ctypes.c_void_p(out.data_ptr()),
                                   current_stream()))
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32).reshape(-1, 4)


def site_normals(seed, sweep, stream, chain, count, precision=FP64, lanes=4):
    """The GPU's update normals of sites 0..count-1 (one chain, one sweep) for a sampler whose
    Philox blocks serve `lanes` chains."""
    import torch

    dt = torch.float32 if precision == FP32 else torch.float64
    out = torch.empty(int(count), dtype=dt, device="cuda")
    _check(lib().gmrf_site_normals(int(seed), sweep, stream, chain, int(lanes), precision, int(count),
                                   ctypes.c_void_p(out.data_ptr()), current_stream()))
    torch.cuda.synchronize()
    return out.cpu().numpy()


class Sampler:
    """A chromatic Gibbs sampler over one or more fields (see include/gmrf.h).

    fields: list of dicts with keys kind, dims, n, y and, for CSR fields, row_ptr, col_idx and
    optionally weights, colors, color_seed; optional per field: x0 ([chains, n]), tau0,
    sigma2_0 and beta0 ([chains]), stream_id (default: the field's index).  intercept=True adds
    the flat-prior intercept beta0 of Sec. 3.1 (initial value beta0_0).  With
    likelihood=LIKELIHOOD_BINOMIAL every field carries `trials` ([n] ints) and y holds the
    successes; beta0 ~ N(beta0_prior) (Sec. 3.2).
    """

    def __init__(self, fields, *, precision=FP32, chains=1, seed=0, prior=PRIOR_ICAR, rho=1.0,
                 a_tau=1.0, b_tau=0.01, a_sigma=1.0, b_sigma=0.01, fix_hyper=False, tau0=1.0,
                 sigma2_0=1.0, start_sweep=0, burn_in=0, thin=1, trace_capacity=4096,
                 algorithm=ALGO_CHROMATIC, graph_sweeps=0, flags=0, stream=None, intercept=False,
                 beta0_0=0.0, likelihood=LIKELIHOOD_GAUSSIAN, beta0_prior=(0.0, 1000.0), tuning=None,
                 autotune_sweeps=30):
        L = lib()
        self._h = ctypes.c_void_p()
        self.chains = int(chains)
        self.fields = fields
        keep = []
        descs = (FieldDesc * len(fields))()
        for i, f in enumerate(fields):
            d = descs[i]
            d.kind = int(f["kind"])
            dims = list(f.get("dims", (0, 0, 0))) + [0, 0, 0]
            for k in range(3):
                d.dims[k] = int(dims[k])
            d.n = int(f["n"])
            arrs = {}
            arrs["y"] = _f64(f["y"])
            if f.get("x0") is not None:
                arrs["x0"] = _f64(np.broadcast_to(np.asarray(f["x0"], np.float64),
                                                  (self.chains, d.n)))
            for key in ("tau0", "sigma2_0", "beta0"):
                if f.get(key) is not None:
                    arrs[key] = _f64(np.broadcast_to(np.asarray(f[key], np.float64), (self.chains,)))
            if d.kind == CSR:
                arrs["row_ptr"] = _i32(f["row_ptr"])
                arrs["col_idx"] = _i32(f["col_idx"])
                if f.get("weights") is not None:
                    arrs["weights"] = _f64(f["weights"])
                if f.get("colors") is not None:
                    arrs["colors"] = _i32(f["colors"])
                d.color_seed = int(f.get("color_seed", 0))
            d.y = _p(arrs["y"], ctypes.c_double)
            d.x0 = _p(arrs.get("x0"), ctypes.c_double)
            d.tau0 = _p(arrs.get("tau0"), ctypes.c_double)
            d.sigma2_0 = _p(arrs.get("sigma2_0"), ctypes.c_double)
            d.beta0 = _p(arrs.get("beta0"), ctypes.c_double)
            if f.get("trials") is not None:
                arrs["trials"] = _i32(f["trials"])
            d.trials = _p(arrs.get("trials"), ctypes.c_int32)
            d.row_ptr = _p(arrs.get("row_ptr"), ctypes.c_int32)
            d.col_idx = _p(arrs.get("col_idx"), ctypes.c_int32)
            d.weights = _p(arrs.get("weights"), ctypes.c_double)
            d.colors = _p(arrs.get("colors"), ctypes.c_int32)
            d.stream_id = int(f.get("stream_id", i))
            keep.append(arrs)
        model = Model(int(prior), float(rho), float(a_tau), float(b_tau), float(a_sigma),
                      float(b_sigma), 1 if fix_hyper else 0, float(tau0), float(sigma2_0),
                      1 if intercept else 0, float(beta0_0), int(likelihood), float(beta0_prior[0]),
                      float(beta0_prior[1]))
        opts = Opts(int(precision), self.chains, int(seed), int(start_sweep), int(burn_in),
                    int(thin), int(trace_capacity), int(algorithm), int(graph_sweeps), int(flags), None)
        self.stream = current_stream() if stream is None else stream
        # tuning: None (the library's cost models), a dict of gmrf_tuning fields, or "auto"
        # (gmrf_autotune on these arguments, cached per process)
        self.tuning_us_per_sweep = None
        tun = None
        if isinstance(tuning, str):
            if tuning != "auto":
                raise ValueError("tuning must be None, a dict or 'auto'")
            tun = Tuning()
            us = ctypes.c_double(0)
            _check(L.gmrf_autotune(descs, len(fields), ctypes.byref(model), ctypes.byref(opts), int(autotune_sweeps),
                                   self.stream, ctypes.byref(tun), ctypes.byref(us)))
            self.tuning_us_per_sweep = us.value
        elif tuning is not None:
            tun = Tuning.from_dict(tuning)
        if tun is not None:
            opts.tuning = ctypes.pointer(tun)
        self.tuning = None if tun is None else tun.to_dict()
        _check(L.gmrf_sampler_create(ctypes.byref(self._h), descs, len(fields), ctypes.byref(model),
                                     ctypes.byref(opts), self.stream))
        self.precision = int(precision)

    def close(self):
        if self._h:
            lib().gmrf_sampler_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def sweep(self, nsweeps=1, with_hyper=True):
        _check(lib().gmrf_sweep(self._h, int(nsweeps), 1 if with_hyper else 0))

    def reset(self):
        _check(lib().gmrf_sampler_reset(self._h))

    def launch_stage(self, stage, accumulate=False):
        """Launch stage `stage` of a sweep once (diagnostic); returns the stage's description."""
        name = ctypes.c_char_p()
        _check(lib().gmrf_launch_stage(self._h, int(stage), 1 if accumulate else 0, ctypes.byref(name)))
        return name.value.decode()

    def debug_poison(self):
        """Mark the sampler as after a CUDA error (later calls raise with GMRF_E_STATE)."""
        _check(lib().gmrf_debug_poison(self._h))

    def hyper_update(self):
        _check(lib().gmrf_hyper_update(self._h))

    def fetch(self, field=0, chain=0, trace=0):
        n = int(self.fields[field]["n"])
        x = np.zeros(n)
        mean = np.zeros(n)
        var = np.zeros(n)
        tt = np.zeros(max(int(trace), 1))
        ts = np.zeros(max(int(trace), 1))
        nt = ctypes.c_int64(0)
        tau = ctypes.c_double(0)
        sig = ctypes.c_double(0)
        _check(lib().gmrf_fetch_samples(self._h, field, chain, _p(x, ctypes.c_double),
                                        _p(mean, ctypes.c_double), _p(var, ctypes.c_double),
                                        int(trace), _p(tt, ctypes.c_double), _p(ts, ctypes.c_double),
                                        ctypes.byref(nt), ctypes.byref(tau), ctypes.byref(sig)))
        m = min(int(trace), nt.value)
        return {"x": x, "mean": mean, "var": var, "tau_trace": tt[:m], "sigma2_trace": ts[:m],
                "n_trace": nt.value, "tau": tau.value, "sigma2": sig.value}

    def fetch_intercept(self, field=0, chain=0, trace=0):
        """Current beta0 and its last `trace` values (oldest first) of one (field, chain)."""
        tb = np.zeros(max(int(trace), 1))
        nt = ctypes.c_int64(0)
        b = ctypes.c_double(0)
        _check(lib().gmrf_fetch_intercept(self._h, field, chain, int(trace), _p(tb, ctypes.c_double),
                                          ctypes.byref(nt), ctypes.byref(b)))
        m = min(int(trace), nt.value)
        return {"beta0": b.value, "beta0_trace": tb[:m], "n_trace": nt.value}

    def trace_diagnostics(self, field=0, param=PARAM_TAU2, n_last=0):
        """IAT (Geyer's initial monotone sequence), ESS per chain and the PSRF over chains of the
        last n_last trace values (0: all) of one parameter, computed on the device."""
        iat = np.zeros(self.chains)
        ess = np.zeros(self.chains)
        ps = ctypes.c_double(0)
        _check(lib().gmrf_trace_diagnostics(self._h, field, int(param), int(n_last), _p(iat, ctypes.c_double),
                                            _p(ess, ctypes.c_double), ctypes.byref(ps)))
        return {"iat": iat, "ess": ess, "psrf": ps.value}

    def site_psrf(self, field=0):
        """Per-site PSRF over chains (natural order) and its maximum."""
        out = np.zeros(int(self.fields[field]["n"]))
        mx = ctypes.c_double(0)
        _check(lib().gmrf_site_psrf(self._h, field, _p(out, ctypes.c_double), ctypes.byref(mx)))
        return out, mx.value

    def fetch_x(self, field=0, chain=0):
        n = int(self.fields[field]["n"])
        x = np.zeros(n)
        _check(lib().gmrf_fetch_samples(self._h, field, chain, _p(x, ctypes.c_double), None, None,
                                        0, None, None, None, None, None))
        return x

    def fetch_mean(self, field=0, chain=0, out=None):
        """Posterior mean of one (field, chain) over the accumulated sweeps, natural order, into
        `out` (a float64 host array of n, e.g. a pinned tensor's numpy view) or a new array."""
        n = int(self.fields[field]["n"])
        m = np.zeros(n) if out is None else out
        if m.dtype != np.float64 or m.shape != (n,) or not m.flags["C_CONTIGUOUS"]:
            raise ValueError(f"out must be a contiguous float64 array of {n}")
        _check(lib().gmrf_fetch_samples(self._h, field, chain, None, _p(m, ctypes.c_double), None,
                                        0, None, None, None, None, None))
        return m

    def fetch_pooled(self, field=0, mean=None, var=None, want_var=True):
        """Posterior mean and variance of one field pooled over its chains, natural order, into
        `mean` / `var` (contiguous float64 host arrays of n, e.g. pinned tensors' numpy views) or
        new arrays; var is None when want_var is false."""
        n = int(self.fields[field]["n"])
        m = np.zeros(n) if mean is None else mean
        v = (np.zeros(n) if var is None else var) if want_var else None
        for a in (m, v):
            if a is not None and (a.dtype != np.float64 or a.shape != (n,) or not a.flags["C_CONTIGUOUS"]):
                raise ValueError(f"outputs must be contiguous float64 arrays of {n}")
        _check(lib().gmrf_fetch_pooled(self._h, field, _p(m, ctypes.c_double), _p(v, ctypes.c_double)))
        return m, v

    def set_data(self, field, y, trials=None, x0=None):
        """Replace one field's observations (and binomial trials, initial states) and restart
        every chain, as a sampler created with these arrays would start."""
        ya = _f64(y)
        ta = _i32(trials)
        # an out-of-range field goes to the library, which rejects it
        n = int(self.fields[field]["n"]) if 0 <= int(field) < len(self.fields) else ya.size
        xa = None if x0 is None else _f64(np.broadcast_to(np.asarray(x0, np.float64), (self.chains, n)))
        if ya.shape != (n,) or (ta is not None and ta.shape != (n,)):
            raise ValueError(f"y and trials must have {n} entries")
        _check(lib().gmrf_sampler_set_data(self._h, int(field), _p(ya, ctypes.c_double), _p(ta, ctypes.c_int32),
                                           _p(xa, ctypes.c_double)))

    def colors(self, field=0):
        n = int(self.fields[field]["n"])
        c = np.zeros(n, np.int32)
        k = ctypes.c_int32(0)
        _check(lib().gmrf_field_colors(self._h, field, _p(c, ctypes.c_int32), ctypes.byref(k)))
        return c, k.value

    def info(self):
        out = Info()
        _check(lib().gmrf_sampler_info(self._h, ctypes.byref(out)))
        return {k: getattr(out, k) for k, _ in Info._fields_}
