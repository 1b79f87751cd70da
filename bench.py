#!/usr/bin/env python3
"""Benchmark of the chromatic Gibbs sampler (site-updates per second) on synthetic workloads.

Default workload: a 256^3 first-order (6-neighbour) intrinsic CAR lattice with the parity
colouring, observations = 50 ellipsoidal activations + N(0, 1) noise, FP32 state with FP64
hyperparameter reductions, 8 chains, 500 sweeps (the first 250 burn-in, the rest accumulated
into the running posterior mean and variance), tau and sigma^2 drawn every sweep.  Its state
(537 MB) and observations (67 MB) live in HBM, so its colour steps are bound by HBM bandwidth.

One step = one complete MCMC run of the workload on device-resident inputs: restart from the
initial state, then all sweeps (every colour step, the fused reductions, the conjugate draws,
the accumulation), replayed as CUDA graphs.  L2 is flushed (a 512 MiB write) between timed
steps, outside the per-step CUDA events.

Printed: one JSON line with the site-update rate, the end-to-end rate through the C ABI with
host buffers, the roofline of the dominant kernel, the FP32-vs-FP64 accuracy of the posterior
means and traces with the speed-up over the plain FP64 sweep at that accuracy, the clocks seen,
and the oracle's CPU rate on a bounded sample.  ``--impl reference`` times the oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1702_05518_gb300 import workloads as wl  # noqa: E402

METRIC = "site-updates/sec & HBM GB/s vs peak: batched FP32 vs plain FP64 chromatic Gibbs"
UNIT = "site-updates/s"


# ----------------------------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------------------------
def workload_spec(name: str):
    """Fields and run parameters of a named workload."""
    if name == "image1024":
        return dict(name="1024x1024 8-neighbour ICAR, 2x2 colouring, 20 Gaussian bumps + N(0,1)",
                    fields=wl.image_1024_bumps(seed=2), chains=1, sweeps=2000, burn_in=1000,
                    prior="icar", rho=1.0, seed=2, graph_sweeps=50, cpu_sweeps=20, acc_sweeps=(2000, 1000),
                    plain_sweeps=200)
    if name == "image64":
        return dict(name="64x64 4-neighbour ICAR, checkerboard, 4-level block image + N(0,0.5^2)",
                    fields=wl.image_64_block(seed=0), chains=1, sweeps=1000, burn_in=500,
                    prior="icar", rho=1.0, seed=0, graph_sweeps=50, cpu_sweeps=1000)
    if name == "volume256":
        return dict(name="256^3 6-neighbour ICAR, parity colouring, 50 ellipsoids + N(0,1), 8 chains",
                    fields=wl.volume_ellipsoids(seed=5), chains=8, sweeps=500, burn_in=250,
                    prior="icar", rho=1.0, seed=5, graph_sweeps=25, cpu_sweeps=1, acc_sweeps=(500, 250),
                    plain_sweeps=40)
    if name in ("delaunay16k", "delaunay16k_ldf"):
        # Jones-Plassmann with random 32-bit priorities, as the workload is stated; the _ldf
        # variant takes the sampler's default order (largest degree first, 6 colours against 7)
        f = wl.delaunay_pcar(seed=3)
        f[0]["color_seed"] = 3
        ldf = name.endswith("_ldf")
        return dict(name="Delaunay 16384 points, proper CAR rho=0.95, 8 chains, JP colouring with "
                    + ("largest-degree-first" if ldf else "random 32-bit") + " priorities", fields=f, chains=8,
                    sweeps=5000, burn_in=2500, prior="pcar", rho=0.95, seed=3, graph_sweeps=50,
                    cpu_sweeps=50, acc_sweeps=(5000, 2500), color_random=not ldf)
    if name == "batched":
        fields = wl.batched_uneven(seed=4)
        for i, f in enumerate(fields):
            f["color_seed"] = 100 + i
        return dict(name="224 lattices (sides log-U[32,512]) + 32 Delaunay graphs (n log-U[1k,50k])",
                    fields=fields, chains=1, sweeps=1000, burn_in=500, prior="icar", rho=1.0,
                    seed=4, graph_sweeps=25, cpu_sweeps=3)
    if name in ("paper50", "paper512"):
        # Sec. 3.1 simulation: p x p image, 5 exp(-|v|^2/2)/pi on [-3, 3]^2, 8-neighbour intrinsic
        # prior, flat intercept, InvGam(0.001, 0.001) on tau^2 and sigma^2, three chains, 10,000
        # iterations with 8,000 burn-in; N(0, 1) noise at p = 50 and N(0, 50^2) at p = 512.
        p, noise = (50, 1.0) if name == "paper50" else (512, 50.0)
        y = (wl.paper_image(p) + wl.rng(6).normal(0.0, noise, (p, p))).ravel()
        f = {"kind": wl.LATTICE2D_8, "dims": (p, p), "n": p * p, "y": y}
        return dict(name=f"{p}x{p} image of Sec. 3.1 (noise sd {noise:g}), 8-neighbour ICAR + intercept, "
                         "InvGam(0.001, 0.001), 3 chains", fields=[f], chains=3, sweeps=10_000, burn_in=8000,
                    prior="icar", rho=1.0, seed=6, graph_sweeps=100, cpu_sweeps=2000 if p == 50 else 20,
                    intercept=True, hyper=dict(a_tau=0.001, b_tau=0.001, a_sigma=0.001, b_sigma=0.001))
    if name == "election":
        # Sec. 3.2 stand-in: 14,926 precinct-like sites on a Delaunay graph, binomial counts with
        # the logistic link (Polya-Gamma augmentation), proper CAR rho 0.995, beta0 ~ N(0, 1000),
        # tau^2 ~ InvGam(1, 1); one chain, 10,000 iterations, the first 5,000 burn-in.
        f = wl.binomial_delaunay(seed=7)
        f[0]["color_seed"] = 7
        return dict(name="Delaunay 14926 sites, binomial counts (trials log-U[1,64], 2.2% missing), logistic "
                         "link + Polya-Gamma, proper CAR rho=0.995, 1 chain", fields=f, chains=1, sweeps=10_000,
                    burn_in=5000, prior="pcar", rho=0.995, seed=7, graph_sweeps=100, cpu_sweeps=20,
                    likelihood="binomial", hyper=dict(a_tau=1.0, b_tau=1.0, beta0_prior=(0.0, 1000.0)))
    raise SystemExit(f"unknown workload {name}")


def site_updates_per_step(spec):
    return sum(f["n"] for f in spec["fields"]) * spec["chains"] * spec["sweeps"]


def colour_classes(field, colors=None):
    """Sites per colour class of a field (closed forms for lattices; CSR from its colouring)."""
    k = field["kind"]
    if k == wl.CSR:
        return np.bincount(colors).tolist()
    if k == wl.LATTICE2D_8:
        H, W = field["dims"][:2]
        return [((H - a + 1) // 2) * ((W - b + 1) // 2) for a in (0, 1) for b in (0, 1)]
    if k == wl.LATTICE3D_6:
        L, H, W = field["dims"]
        even = (L * H * W + 1) // 2
        return [even, L * H * W - even]
    H, W = field["dims"][:2]
    even = (H * W + 1) // 2
    return [even, H * W - even]


def _stage_fields(spec, stage_name, colour, colourings):
    """The fields a launch of the named stage covers: (index, field, its sites in the launch,
    its colour-class sizes)."""
    for fi, f in enumerate(spec["fields"]):
        kind = f["kind"]
        cls = colour_classes(f, colourings.get(fi))
        if "fused" in stage_name:
            if ("8-neighbour" in stage_name) != (kind == wl.LATTICE2D_8) or kind not in (wl.LATTICE2D_4, wl.LATTICE2D_8):
                continue
            yield fi, f, f["n"], cls
            continue
        if "colour step" not in stage_name:
            continue
        if ("CSR" in stage_name) != (kind == wl.CSR):
            continue
        if kind != wl.CSR and ("3-D" in stage_name) != (kind == wl.LATTICE3D_6):
            continue
        if colour >= len(cls):
            continue
        yield fi, f, cls[colour], cls


def bytes_per_update(field, chains, cls, S=4):
    """Least HBM bytes per site-update of the method (each state value written once per sweep,
    each other-colour neighbour value read once per colour step, the observations read once per
    sweep and shared by the chains, the reductions fused, accumulation off):
        2-colour lattices (2-D 4-neighbour, 3-D 6-neighbour): 2 S + S / C;
        4-colour 8-neighbour lattice: 4 S + S / C;
        CSR graph with k colours and mean degree deg: k S + (S + 4 (deg + 1)) / C
    (row pointer and column indices at 4 bytes), with S the bytes of a state value."""
    C = chains
    if field["kind"] == wl.CSR:
        deg = float(field["row_ptr"][-1]) / max(1, field["n"])
        return len(cls) * S + (S + 4 * (deg + 1)) / C
    k = 4 if field["kind"] == wl.LATTICE2D_8 else 2
    return k * S + S / C


def stage_algorithmic_bytes(spec, stage_name, colour, colourings, S=4):
    """Algorithmic bytes of one launch of the stage: its site-updates times bytes_per_update."""
    C = spec["chains"]
    return sum(units * C * bytes_per_update(f, C, cls, S)
               for _, f, units, cls in _stage_fields(spec, stage_name, colour, colourings))


def stage_design_bytes(spec, stage_name, colour, colourings, S=4):
    """Least bytes the kernel design itself must move per launch (accumulation off), summed over
    its fields:
    fused 2-D sweep (all colours in one launch, state staged in shared memory): every site's
    state read once and written once, y read once: n (2 C S + S);
    lattice colour step c: the other colours' states read once, y and the new state of class c:
        (n - n_c) C S + n_c S + n_c C S;
    CSR colour step c: for the sites of class c, row pointers, degrees, permutation, y, the
    column indices of their edges, the states of the distinct neighbours, and the new states.
    """
    C = spec["chains"]
    total = 0
    for fi, f, n_c, cls in _stage_fields(spec, stage_name, colour, colourings):
        if "fused" in stage_name:
            total += f["n"] * (2 * C * S + S)
        elif f["kind"] == wl.CSR:
            col = colourings[fi]
            rp, ci = f["row_ptr"], f["col_idx"]
            members = np.flatnonzero(col == colour)
            deg = np.diff(rp)[members]
            nbrs = np.unique(np.concatenate([ci[rp[i]:rp[i + 1]] for i in members])) if len(members) else []
            total += n_c * (4 + S + 4 + S) + 4 * int(deg.sum()) + len(nbrs) * C * S + n_c * C * S
        else:
            total += (sum(cls) - n_c) * C * S + n_c * S + n_c * C * S
    return total


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant kernel of
# a workload, from one ncu capture (cold L2: ncu flushes caches before the launch), with the
# SHA-256 of what the kernel is compiled from at capture time: its source files and, for the
# shared header, the text of its argument struct ("file:Struct").  Reported only while those are
# unchanged.
MEASURED_TRAFFIC = {
    "volume256": dict(kernel="lattice3d_kernel<2, 1, 0, 0>", bytes=331_137_536 + 235_047_680,
                      sources={"lattice3d.cu": "a6cfedab49ce2a4f8b102bbac80e5a0a24dcc2bbb99044e0a03df17ad372ae97",
                               "gmrf_device.cuh": "aed73d1682b3c1b60aeb41a9226e07ca5a05172953ac21a6ebf5cf66c269fb52",
                               "gmrf_internal.h:StepArgs": "f1074e9506e5570bccaa0fa63d2106830a8bbbd7d9a256d2de0630bbe74378c7"}),
}


def _source_digest(spec: str):
    """SHA-256 of a kernel source file, or of one struct's text in it ("file:Struct")."""
    import hashlib

    name, _, struct = spec.partition(":")
    path = os.path.join(ROOT, "paper_1702_05518_gb300", "csrc", name)
    data = open(path, "rb").read()
    if struct:
        text = data.decode()
        i = text.index("struct " + struct + " {")
        data = text[i:text.index("\n};", i) + 3].encode()
    return hashlib.sha256(data).hexdigest()


def measured_traffic(workload: str):
    """DRAM bytes per launch of the workload's dominant kernel, or None if not captured for the
    current kernel sources."""
    rec = MEASURED_TRAFFIC.get(workload)
    if rec is None:
        return None
    for spec, digest in rec["sources"].items():
        try:
            if _source_digest(spec) != digest:
                return None
        except (OSError, ValueError):
            return None
    return rec["bytes"]


# ----------------------------------------------------------------------------------------------
# Clocks
# ----------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while active."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------------------------
# CPU baseline: the oracle on a bounded sample of the workload
# ----------------------------------------------------------------------------------------------
def oracle_rate(spec, sweeps):
    import oracle
    from paper_1702_05518_gb300.workloads import CSR

    kinds = {wl.LATTICE2D_4: oracle.LAT2D_4, wl.LATTICE2D_8: oracle.LAT2D_8, wl.LATTICE3D_6: oracle.LAT3D_6}
    prepared = []
    for i, f in enumerate(spec["fields"]):
        if f["kind"] == CSR:
            graph = (f["row_ptr"], f["col_idx"])
            colors = oracle.color_graph(f["row_ptr"], f["col_idx"], f.get("color_seed", 0),
                                        ldf=not spec.get("color_random", False))[0]
        else:
            graph = oracle.lattice_csr(kinds[f["kind"]], f["dims"])
            colors = oracle.lattice_colors(kinds[f["kind"]], f["dims"])[0]
        prepared.append((graph, colors, f["y"], i))
    t0 = time.perf_counter()
    updates = 0
    for graph, colors, y, i in prepared:
        st = oracle.initial_state(y, spec["chains"])
        hp = spec.get("hyper", {})
        hp = {("a_sig" if k == "a_sigma" else "b_sig" if k == "b_sigma" else k): v for k, v in hp.items()}
        if spec.get("likelihood") == "binomial":
            hp["trials"] = spec["fields"][i]["trials"]
            st = oracle.initial_state(y, spec["chains"], x0=np.zeros(len(y)))
        oracle.run(graph, colors, y, st, seed=spec["seed"], nsweeps=sweeps, stream=i, prior=spec["prior"],
                   intercept=spec.get("intercept", False), **hp,
                   rho=spec["rho"], burn_in=0, accumulate=True)
        updates += len(y) * spec["chains"] * sweeps
    dt = time.perf_counter() - t0
    return updates / dt, dt, updates


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return platform.processor() or platform.machine()


# ----------------------------------------------------------------------------------------------
# Distributed helpers (one process per GPU; replicas with independent seeds, no data exchange)
# ----------------------------------------------------------------------------------------------
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_seed(base_seed: int, rank: int) -> int:
    """Each rank runs an independent replica: a different Philox key per rank."""
    return int(base_seed) + 1000003 * int(rank)


def max_over_ranks(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# ----------------------------------------------------------------------------------------------
# Arms
# ----------------------------------------------------------------------------------------------
def reference_sample(spec, budget=2e7):
    """The workload cut to a bounded sample for the oracle's timed steps: a 3-D lattice larger
    than `budget` site-updates per sweep keeps its first planes (the same lattice, fewer planes;
    the oracle's work per site-update does not depend on the extent), other fields stay whole."""
    fields = spec["fields"]
    C = spec["chains"]
    if len(fields) == 1 and fields[0]["kind"] == wl.LATTICE3D_6 and fields[0]["n"] * C > budget:
        f = fields[0]
        L, H, W = f["dims"]
        planes = max(2, int(budget // (H * W * C)))
        n = planes * H * W
        cut = dict(f, dims=(planes, H, W), n=n, y=np.ascontiguousarray(f["y"][:n]))
        cut.pop("truth", None)
        return dict(spec, fields=[cut]), f"the first {planes} of {L} planes ({planes}x{H}x{W} sites)"
    return spec, "the whole workload"


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    spec, part = reference_sample(workload_spec(args.workload))
    sample = max(1, spec["cpu_sweeps"] // 4) if args.workload != "image64" else 100
    for _ in range(args.warmup):
        oracle_rate(spec, sample)
    times = []
    updates = 0
    for _ in range(args.steps):
        _, dt, u = oracle_rate(spec, sample)
        times.append(dt)
        updates += u
    value = updates / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": spec["name"], "sample": f"{sample} sweeps of {part} per step",
                       "chains": spec["chains"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{sample} sweeps of {part} per step, {args.steps} steps; CPU: {cpu_model()}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def sampler_kwargs(spec, g, seed, **over):
    """Sampler arguments of a workload: FP32 state, its prior, chains, intercept and priors."""
    kw = dict(precision=g.FP32, chains=spec["chains"], seed=seed,
              prior=g.PRIOR_PCAR if spec["prior"] == "pcar" else g.PRIOR_ICAR, rho=spec["rho"],
              burn_in=spec["burn_in"], graph_sweeps=spec["graph_sweeps"], trace_capacity=spec["sweeps"],
              intercept=spec.get("intercept", False), **spec.get("hyper", {}))
    if spec.get("likelihood") == "binomial":
        kw["likelihood"] = g.LIKELIHOOD_BINOMIAL
    if spec.get("color_random"):
        kw["flags"] = g.FLAG_COLOR_RANDOM
    kw.update(over)
    return kw


def run_profile_case(args):
    """A fixed launch sequence for a profiler: create, S sweeps launched stage by stage, fetch."""
    import torch

    from paper_1702_05518_gb300 import build as libbuild
    from paper_1702_05518_gb300 import gmrf as g

    torch.cuda.set_device(0)
    if not os.path.exists(g.LIB_PATH):
        libbuild.build()
    spec = workload_spec(args.workload)
    with g.Sampler(spec["fields"], **sampler_kwargs(spec, g, spec["seed"], graph_sweeps=0)) as s:
        s.sweep(args.profile_sweeps)
        x = s.fetch_x(0, 0)
        info = s.info()
    print(json.dumps({"profile_case": spec["name"], "sweeps": args.profile_sweeps,
                      "launches_per_sweep": info["launches_per_sweep"], "finite": bool(np.isfinite(x).all())}))
    return 0


def accuracy_block(spec, g, seed):
    """Accuracy of the FP32 sampler against FP64 on the workload (one field).

    Both run the same chains (same seed and Philox counters, so they are coupled draw for draw)
    for acc_sweeps sweeps, the first acc_burn of them burn-in: the FP32 sampler of the benchmark
    and the FP64 sampler (which agrees with the oracle within 1e-12, and with the plain FP64 sweep
    to rounding).  Reported: the largest errors of the FP32 posterior means, final states and
    tau / sigma^2 traces relative to max(|FP64 value|, 1) (traces: relative to the value), and
    the Monte Carlo standard error of each FP64 posterior mean, i.e. the statistical error of the
    estimate itself: with two or more chains the standard deviation over the chains of their
    means (each chain's mean is an independent estimate), with one chain sqrt(var tau_int / N)
    with the integrated autocorrelation time of the tau^2 chain.  The FP32 sampler counts as
    equally accurate when every error of a chain's posterior mean is below that site's standard
    error."""
    import torch

    T, burn = spec["acc_sweeps"]
    f0 = spec["fields"][0]
    n, C = f0["n"], spec["chains"]
    runs = {}
    for prec in (g.FP32, g.FP64):
        s = g.Sampler(spec["fields"], **sampler_kwargs(spec, g, seed, precision=prec, burn_in=burn,
                                                       trace_capacity=T))
        s.sweep(T)
        torch.cuda.synchronize()
        runs[prec] = s
    s32, s64 = runs[g.FP32], runs[g.FP64]
    N = T - burn
    # standard error of each FP64 posterior mean
    if C >= 2:
        sm = np.zeros(n)
        sq = np.zeros(n)
        for c in range(C):
            m = s64.fetch(0, c)["mean"]
            sm += m
            sq += m * m
        var_between = np.maximum(sq - sm * sm / C, 0.0) / (C - 1)
        se = np.sqrt(var_between)
        se_kind = f"std over the {C} chains of their posterior means"
    else:
        iat = float(s64.trace_diagnostics(0, g.PARAM_TAU2, N)["iat"][0])
        se = np.sqrt(s64.fetch(0, 0)["var"] * iat / N)
        se_kind = f"sqrt(var tau_int / N), tau_int = {iat:.1f} (tau^2 chain), N = {N}"
    worst = {"mean": 0.0, "x": 0.0, "tau_trace": 0.0, "sigma2_trace": 0.0}
    ratio = 0.0
    for c in range(C):
        a = s32.fetch(0, c, trace=T)
        b = s64.fetch(0, c, trace=T)
        d = np.abs(a["mean"] - b["mean"])
        worst["mean"] = max(worst["mean"], float(np.max(d / np.maximum(np.abs(b["mean"]), 1.0))))
        worst["x"] = max(worst["x"], float(np.max(np.abs(a["x"] - b["x"]) / np.maximum(np.abs(b["x"]), 1.0))))
        for key in ("tau_trace", "sigma2_trace"):
            worst[key] = max(worst[key], float(np.max(np.abs(a[key] - b[key]) / np.abs(b[key]))))
        ratio = max(ratio, float(np.max(d / np.maximum(se, 1e-300))))
    s32.close()
    s64.close()
    return {"sweeps": T, "burn_in": burn, "reference": "FP64 sampler, same chains (coupled)",
            "mean_max_relerr": worst["mean"], "x_max_relerr": worst["x"],
            "tau_trace_max_relerr": worst["tau_trace"], "sigma2_trace_max_relerr": worst["sigma2_trace"],
            "mc_se_median": float(np.median(se)), "mc_se_min": float(np.min(se)), "mc_se": se_kind,
            "mean_err_over_se_max": ratio, "equal_accuracy": bool(ratio < 1.0)}


def run_ours(args):
    import torch

    from paper_1702_05518_gb300 import build as libbuild
    from paper_1702_05518_gb300 import gmrf as g

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if not os.path.exists(g.LIB_PATH):
        libbuild.build()
    spec = workload_spec(args.workload)
    seed = replica_seed(spec["seed"], rank)
    kw = sampler_kwargs(spec, g, seed)
    if getattr(args, "tune", False):
        kw["tuning"] = "auto"
        kw["autotune_sweeps"] = max(10, min(100, spec["graph_sweeps"] or 10))
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    units = site_updates_per_step(spec)

    s = g.Sampler(spec["fields"], **kw)
    tuned = s.tuning if kw.get("tuning") == "auto" else None
    info = s.info()
    for _ in range(args.warmup):
        s.reset()
        s.sweep(spec["sweeps"])
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(k & 0xFF)  # evict the previous step's data from L2 (untimed)
            starts[k].record(stream)
            s.reset()
            s.sweep(spec["sweeps"])
            ends[k].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        wall = time.perf_counter() - w0
    clocks = clk.summary()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    dev_s = sum(step_ms) / 1e3
    dev_s_max = max_over_ranks(dev_s, world, device="cuda")
    value = world * units * args.steps / dev_s_max

    # Statistical efficiency of the last timed run (Sec. 3.1): IAT and ESS of the tau^2 chains
    # over the retained sweeps, on the device, and the cost per effective sample
    # CES = kappa T / N with T the run's time; pooled over the chains: T / sum of their ESS.
    efficiency = None
    retained = spec["sweeps"] - spec["burn_in"]
    if len(spec["fields"]) == 1 and retained >= 4:
        t_run = dev_s / args.steps
        efficiency = {"retained": retained, "run_s": t_run}
        params = [("tau^2", g.PARAM_TAU2)]
        if spec.get("intercept") or spec.get("likelihood") == "binomial":
            params.append(("beta0", g.PARAM_BETA0))
        for label, pid in params:
            d = s.trace_diagnostics(0, pid, retained)
            efficiency[label] = {"iat": [float(v) for v in d["iat"]], "ess": [float(v) for v in d["ess"]],
                                 "psrf": None if d["psrf"] != d["psrf"] else float(d["psrf"]),
                                 "ces_s": t_run / float(np.sum(d["ess"]))}

    # Resident samplers (a small single 2-D lattice, a single graph below 32768 sites, or the quad
    # lattice's tiles in one wave): a batch of sweeps is two launches (the unit-rate Gamma variates,
    # with the batch's normals where the resident kernel does not draw its own, then the resident
    # kernel); timed as whole batches.
    resident_batch = None
    if info["resident"]:
        G = spec["graph_sweeps"]
        rb = min(128, max(64, G))
        nb = min(rb, G) if G > 0 else rb
        ev_a, ev_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.reset()
        s.sweep(nb)
        torch.cuda.synchronize()
        ev_a.record(stream)
        for _ in range(10):
            s.sweep(nb)
        ev_b.record(stream)
        torch.cuda.synchronize()
        batch_us = ev_a.elapsed_time(ev_b) * 1e3 / 10
        resident_batch = {"sweeps": nb, "us": batch_us}

    # Each stage of a sweep timed in its place: whole sweeps launched stage by stage in sweep order
    # (accumulation off), CUDA events on the launching stream around every launch, averaged over
    # the sweeps, so each kernel sees the L2 contents its predecessor leaves; the dominant stage is
    # the longest one that moves the state.
    reps = 50
    colourings = {fi: s.colors(fi)[0] for fi, f in enumerate(spec["fields"]) if f["kind"] == wl.CSR}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nst = info["launches_per_sweep"]
    names, colour_of_stage, seen = [], {}, {}
    for st in range(nst):
        names.append(s.launch_stage(st))
        colour_of_stage[st] = seen.get(names[st], 0)
        seen[names[st]] = colour_of_stage[st] + 1
    evs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nst)]
           for _ in range(reps)]
    torch.cuda.synchronize()
    for r in range(reps):
        for st in range(nst):
            evs[r][st][0].record(stream)
            s.launch_stage(st)
            evs[r][st][1].record(stream)
    torch.cuda.synchronize()
    stages = [(st, names[st], sum(evs[r][st][0].elapsed_time(evs[r][st][1]) for r in range(reps)) * 1e3 / reps)
              for st in range(nst)]
    # the roofline is taken on the longest state-moving stage (not the parameter draws)
    movers = [st_ for st_ in stages if "draw" not in st_[1]] or stages
    dom = max(movers, key=lambda x: x[2])
    kernel_us = dom[2]
    algo_bytes = stage_algorithmic_bytes(spec, dom[1], colour_of_stage[dom[0]], colourings)
    design_bytes = stage_design_bytes(spec, dom[1], colour_of_stage[dom[0]], colourings)
    s.close()
    # The random numbers alone of the dominant 3-D colour step (same counters and arithmetic, no
    # state traffic): a floor under the kernel's time like the HBM roofline's.
    rng_only = None
    if "3-D" in dom[1] and "all chains" in dom[1]:
        n_c = sum(units for _, _, units, _ in _stage_fields(spec, dom[1], colour_of_stage[dom[0]], colourings))
        rng_only = g.normals_timing(seed, n_c, spec["chains"], reps=20)

    # The plain single-field FP64 sweep (natural layout, one unfused pass per colour) on the same
    # workload and chains, a bounded number of sweeps: the speed-up of the path is value / its rate.
    plain = None
    if len(spec["fields"]) == 1 and not spec.get("intercept", False) and spec.get("likelihood") != "binomial":
        ps = min(spec["sweeps"], spec.get("plain_sweeps", 200))
        with g.Sampler(spec["fields"], **sampler_kwargs(spec, g, seed, precision=g.FP64, algorithm=g.ALGO_PLAIN,
                                                       graph_sweeps=min(spec["graph_sweeps"], ps))) as sp:
            sp.sweep(ps)
            torch.cuda.synchronize()
            sp.reset()
            ev0.record(stream)
            sp.sweep(ps)
            ev1.record(stream)
            torch.cuda.synchronize()
            prate = spec["fields"][0]["n"] * spec["chains"] * ps / (ev0.elapsed_time(ev1) * 1e-3)
        plain = {"value": prate, "unit": UNIT, "dtype": "f64", "sweeps": ps, "speedup": None}

    # End to end through the C ABI with host buffers.  Serving: one sampler built for the graph
    # (outside the timed region); per step the observations (and trials) go up from pinned host
    # memory (gmrf_sampler_set_data, which also restarts the chains), all sweeps run, and the
    # posterior mean and variance pooled over the chains come back into pinned host memory.  Cold:
    # the same plus creating and destroying the sampler (colouring, layout, tiles, graph capture)
    # inside every step.
    e2e_steps = max(1, min(5, args.steps))
    n_total = sum(f["n"] for f in spec["fields"])
    binom = spec.get("likelihood") == "binomial"
    host_y = [torch.from_numpy(np.ascontiguousarray(f["y"], np.float64)).pin_memory() for f in spec["fields"]]
    host_m = [torch.from_numpy(np.ascontiguousarray(f["trials"], np.int32)).pin_memory() if binom else None
              for f in spec["fields"]]
    host_mean = [torch.empty(f["n"], dtype=torch.float64, pin_memory=True) for f in spec["fields"]]
    host_var = [torch.empty(f["n"], dtype=torch.float64, pin_memory=True) for f in spec["fields"]]
    h2d = (8 + (4 if binom else 0)) * n_total
    d2h = 16 * n_total

    def e2e_step(sampler):
        for fi in range(len(spec["fields"])):
            sampler.set_data(fi, host_y[fi].numpy(), None if host_m[fi] is None else host_m[fi].numpy())
        sampler.sweep(spec["sweeps"])
        for fi in range(len(spec["fields"])):
            sampler.fetch_pooled(fi, mean=host_mean[fi].numpy(), var=host_var[fi].numpy())

    with g.Sampler(spec["fields"], **kw) as s2:
        e2e_step(s2)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step_ms = []
        for _ in range(e2e_steps):
            t1 = time.perf_counter()
            e2e_step(s2)  # ends with the pooled read-back, which synchronises the stream
            e2e_step_ms.append(1e3 * (time.perf_counter() - t1))
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, world, device="cuda")
    e2e_value = world * units * e2e_steps / e2e_s
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        with g.Sampler(spec["fields"], **kw) as s2:
            e2e_step(s2)
    torch.cuda.synchronize()
    cold_s = max_over_ranks(time.perf_counter() - t0, world, device="cuda")
    e2e_cold = world * units * e2e_steps / cold_s

    accuracy = None
    if plain is not None and spec.get("acc_sweeps"):
        accuracy = accuracy_block(spec, g, seed)

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs")
    peak_note = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    achieved = algo_bytes / (kernel_us * 1e-6) / 1e9
    f0 = spec["fields"][0]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": measured_traffic(args.workload), "peak_source": peak_note,
                "kernel": dom[1], "algorithmic_bytes_per_launch": algo_bytes,
                "bytes_per_update": bytes_per_update(f0, spec["chains"],
                                                     colour_classes(f0, colourings.get(0))),
                "avg_launch_us": kernel_us,
                "design_bytes_per_launch": design_bytes,
                "design_frac": design_bytes / (kernel_us * 1e-6) / 1e9 / hbm,
                "normals_only_us": rng_only,
                "normals_only_frac": None if rng_only is None else algo_bytes / (rng_only * 1e-6) / 1e9 / hbm,
                "stages_us": {f"{st}:{name}": round(us, 3) for st, name, us in stages}}
    if resident_batch and info["resident"] in (3, 4):
        # The quad kernel's or the fused sweep's tiles kept in shared memory for a batch of sweeps (one cooperative
        # launch, a grid barrier per sweep): the method's least bytes per sweep (bytes_per_update
        # per site-update, every sweep) over the batch's time, Gamma-variate launch included.
        nb = resident_batch["sweeps"]
        q_bytes = algo_bytes * nb
        ach = q_bytes / (resident_batch["us"] * 1e-6) / 1e9
        roofline = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                    "traffic": None, "peak_source": peak_note,
                    "kernel": "resident batch: Gamma variates, "
                              + ("lattice_quad_resident_kernel" if info["resident"] == 3 else "lattice_fused_resident")
                              + " (cooperative, one block per tile)",
                    "algorithmic_bytes_per_launch": q_bytes,
                    "bytes_per_update": bytes_per_update(f0, spec["chains"], colour_classes(f0)),
                    "avg_launch_us": resident_batch["us"], "sweeps_per_launch": nb,
                    "us_per_sweep": resident_batch["us"] / nb,
                    "note": "the state stays in shared memory and L2 between sweeps, so the bound is the "
                            "latency of a sweep (colour steps, grid barrier, draws), not HBM",
                    "per_sweep_path_stages_us": {f"{st}:{name}": round(us, 3) for st, name, us in stages}}
    elif resident_batch:
        # The resident kernel keeps the chain in shared memory for the whole batch: its HBM bytes
        # per batch are one read and one write of state, mean and M2, one read of y, and the
        # batch's normals (written by their producer, read once), so the bound is the latency of
        # a sweep (colour steps, barriers, the draws), not a roofline; the figures say so.
        nb = resident_batch["sweeps"]
        n = spec["fields"][0]["n"]
        C = spec["chains"]
        res_bytes = 4 * (n * C * 6 + n + 2 * nb * n * C)
        ach = res_bytes / (resident_batch["us"] * 1e-6) / 1e9
        graph = info["resident"] == 2
        roofline = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                    "traffic": None, "peak_source": peak_note,
                    "kernel": "resident batch: Gamma variates, normals, "
                              + ("csr_resident_kernel" if graph else "lattice_resident_kernel"),
                    "algorithmic_bytes_per_launch": res_bytes, "avg_launch_us": resident_batch["us"],
                    "sweeps_per_launch": nb, "us_per_sweep": resident_batch["us"] / nb,
                    "note": "latency-bound (whole sweeps in shared memory, "
                            + ("a cluster of blocks" if graph else "one block") + " per chain): the HBM "
                            "fraction only counts the batch's staging and normals",
                    "per_sweep_path_stages_us": {f"{st}:{name}": round(us, 3) for st, name, us in stages}}

    if rank != 0:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return 0

    cpu = None
    if world == 1 and not args.no_cpu:
        rate, dt, u = oracle_rate(spec, spec["cpu_sweeps"])
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{spec['cpu_sweeps']} sweeps of the full workload ({u} site-updates, {dt:.1f} s); "
                         f"CPU: {cpu_model()}"}
    # per step: every stage of every sweep, one Gamma-variate batch per 64 (or graph_sweeps)
    # sweeps, and the restart kernel; resident samplers: two launches per batch of sweeps (a
    # graph of graph_sweeps sweeps holds ceil(graph_sweeps / batch) batches, a left-over sweep one)
    batch = max(64, spec["graph_sweeps"])
    launches = args.steps * (spec["sweeps"] * info["launches_per_sweep"] + -(-spec["sweeps"] // batch) + 1)
    if info["resident"]:
        G = spec["graph_sweeps"]
        rb = min(128, max(64, G))
        full, rem = divmod(spec["sweeps"], G) if G > 0 else (0, spec["sweeps"])
        chunks = full * -(-G // rb) + (rem if G > 0 else -(-rem // rb))
        # two launches per batch: the Gamma variates (with the batch's normals, except for quad
        # tiles, whose blocks draw their own) and the resident kernel
        launches = args.steps * (2 * chunks + 1)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dev_s_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": spec["name"], "chains": spec["chains"], "sweeps_per_step": spec["sweeps"],
                       "burn_in": spec["burn_in"], "sites": n_total, "graph_sweeps": spec["graph_sweeps"],
                       "l2": "flushed between steps (512 MiB write), outside the timed events",
                       "parallelism": f"replicas x{world}",
                       "launch_config": "autotuned: " + json.dumps(tuned) if tuned else "cost models"},
            "wall_ms_per_step": 1e3 * wall / args.steps,
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps,
                    "step_ms": [round(v, 3) for v in e2e_step_ms],
                    "step_spread": (max(e2e_step_ms) - min(e2e_step_ms)) / (sum(e2e_step_ms) / len(e2e_step_ms)),
                    "per_step": "observations H2D (pinned) + restart, all sweeps, posterior mean and variance "
                                "pooled over the chains D2H (pinned); sampler built once outside the timed region",
                    "cold_value": e2e_cold,
                    "cold_per_step": "the same with sampler creation and destruction inside every step"},
            "gpu_launches": launches,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "plain_fp64": plain,
            "accuracy": accuracy,
            "speedup_equal_accuracy": None,
            "efficiency": efficiency}
    if plain:
        plain["speedup"] = value / plain["value"]
        if accuracy and accuracy["equal_accuracy"]:
            line["speedup_equal_accuracy"] = value / plain["value"]
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="volume256",
                    choices=["image1024", "image64", "volume256", "delaunay16k", "delaunay16k_ldf", "batched", "paper50",
                             "paper512", "election"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--tune", action="store_true",
                    help="launch configuration by gmrf_autotune (measured on this GPU, untimed) instead of the "
                         "library's cost models")
    ap.add_argument("--profile-sweeps", type=int, default=0, metavar="S",
                    help="untimed: run S sweeps of the workload with one launch per stage (no graphs) "
                         "and exit; a short, fixed launch sequence for a profiler to capture")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_sweeps > 0:
        return run_profile_case(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
