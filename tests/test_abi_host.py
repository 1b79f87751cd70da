"""Host-side checks of the C-ABI library (CPU only, no GPU work): the library loads and exports
every entry point include/gmrf.h declares; CSR validation and argument checks reject bad
input before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1702_05518_gb300 import gmrf as g
from paper_1702_05518_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1702_05518_gb300 import build

    build.build()
    return g.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(gmrf_[a-z0-9_]+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(L):
    declared = _declared()
    assert {"gmrf_color_graph", "gmrf_sampler_create", "gmrf_sweep", "gmrf_hyper_update",
            "gmrf_fetch_samples"} <= declared
    for name in declared:
        assert hasattr(L, name), name
    assert set(g.EXPORTED) == declared
    assert L.gmrf_version().decode().count(".") == 2


def test_validate_csr_accepts_graphs_and_counts_components(L):
    rp, ci, _ = wl.delaunay_graph(400, wl.rng(1))
    assert g.validate_csr(rp, ci) == oracle.components(rp, ci) == 1
    e = np.array([[0, 1], [2, 3], [3, 4]])
    rp2, ci2 = wl.csr_from_edges(7, e)
    assert g.validate_csr(rp2, ci2) == oracle.components(rp2, ci2) == 4


@pytest.mark.parametrize("case", ["asym", "self", "dup", "range", "wneg", "wasym", "rp0", "rpdec"])
def test_validate_csr_rejects(L, case):
    rp, ci = wl.cycle_graph(5)
    rp, ci = rp.copy(), ci.copy()
    w = None
    if case == "asym":
        ci[0] = 2 if ci[0] != 2 else 3
    elif case == "self":
        ci[0] = 0
    elif case == "dup":
        ci[1] = ci[0]
    elif case == "range":
        ci[0] = 7
    elif case == "wneg":
        w = np.ones(len(ci))
        w[3] = -1.0
    elif case == "wasym":
        w = np.ones(len(ci))
        w[0] = 2.0
    elif case == "rp0":
        rp[0] = 1
    elif case == "rpdec":
        rp[2] = rp[1] - 1
    with pytest.raises(g.GmrfError) as ex:
        g.validate_csr(rp, ci, w)
    assert ex.value.status == g.E_INVALID


def _lat(n=4):
    return {"kind": wl.LATTICE2D_4, "dims": (n, n, 0), "n": n * n, "y": np.zeros(n * n)}


@pytest.mark.parametrize("bad", ["chains0", "chains65", "thin0", "trace0", "rho1", "ashape", "brate",
                                 "sig0", "dims", "yinf", "colors", "plain_multi", "plain_fp32"])
def test_create_rejects_before_any_cuda_call(L, bad):
    kw = {}
    fields = [_lat()]
    if bad == "chains0":
        kw["chains"] = 0
    elif bad == "chains65":
        kw["chains"] = 65
    elif bad == "thin0":
        kw["thin"] = 0
    elif bad == "trace0":
        kw["trace_capacity"] = 0
    elif bad == "rho1":
        kw.update(prior=g.PRIOR_PCAR, rho=1.0)
    elif bad == "ashape":
        kw["a_tau"] = 0.0
    elif bad == "brate":
        kw["b_sigma"] = -1.0
    elif bad == "sig0":
        kw["sigma2_0"] = 0.0
    elif bad == "dims":
        fields[0]["n"] = 15
    elif bad == "yinf":
        fields[0]["y"] = np.full(16, np.inf)
    elif bad == "colors":
        rp, ci = wl.path_graph(4)
        fields = [{"kind": wl.CSR, "n": 4, "y": np.zeros(4), "row_ptr": rp, "col_idx": ci,
                   "colors": np.zeros(4, np.int32)}]
    elif bad == "plain_multi":
        fields = [_lat(), _lat()]
        kw.update(algorithm=g.ALGO_PLAIN, precision=g.FP64)
    elif bad == "plain_fp32":
        kw.update(algorithm=g.ALGO_PLAIN, precision=g.FP32)
    with pytest.raises(g.GmrfError) as ex:
        g.Sampler(fields, stream=None, **kw)
    assert ex.value.status in (g.E_INVALID, g.E_UNSUPPORTED)
    assert len(g.lib().gmrf_last_error()) > 0


def test_null_arguments(L):
    assert L.gmrf_sweep(None, 1, 1) == g.E_INVALID
    assert L.gmrf_hyper_update(None) == g.E_INVALID
    assert L.gmrf_sampler_info(None, None) == g.E_INVALID
    out = ctypes.c_void_p(1)
    assert L.gmrf_sampler_create(ctypes.byref(out), None, 0, None, None, None) == g.E_INVALID
    assert out.value is None
    L.gmrf_sampler_destroy(None)


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes structures of the binding have the C structures' sizes and field offsets
    (compiled from include/gmrf.h with the host C compiler)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    pairs = {"gmrf_field_desc": g.FieldDesc, "gmrf_model": g.Model, "gmrf_tuning": g.Tuning,
             "gmrf_opts": g.Opts, "gmrf_info": g.Info}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "gmrf.h"', "int main(void) {"]
    for cname, cls in pairs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.run([cc, "-std=c11", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_noalloc_wrapper_checks_tensors_before_any_call():
    # a colors tensor shorter than n (or the wrong type) is refused on the host: the library would
    # write n entries through its pointer
    torch = pytest.importorskip("torch")
    rp, ci = wl.cycle_graph(6)
    rpt = torch.from_numpy(rp.astype(np.int32))
    cit = torch.from_numpy(ci.astype(np.int32))
    with pytest.raises(ValueError, match="colors has 5 elements"):
        g.color_graph_noalloc(rpt, cit, torch.empty(5, dtype=torch.int32))
    with pytest.raises(ValueError, match="colors must be"):
        g.color_graph_noalloc(rpt, cit, torch.empty(6, dtype=torch.int64))
    with pytest.raises(ValueError, match="priorities has 3 elements"):
        g.color_graph_noalloc(rpt, cit, torch.empty(6, dtype=torch.int32), priorities=torch.zeros(3, dtype=torch.int32))
    with pytest.raises(ValueError, match="current CUDA device"):  # host tensors are not device arrays
        g.color_graph_noalloc(rpt, cit, torch.empty(6, dtype=torch.int32))


def test_debug_hooks_reject_bad_arguments(L):
    assert L.gmrf_debug_fail_alloc(-1) == g.E_INVALID
    assert L.gmrf_debug_fail_alloc(0) == g.OK
    assert L.gmrf_debug_poison(None) == g.E_INVALID
