"""gmrf_color_graph_noalloc: the JP colouring with its scratch in a static device array.

Called through the C ABI on device-resident CSR graphs, twice in a row, it must give the
colouring of gmrf_color_graph bit for bit (integer work); sizes above its static capacity and
malformed CSR structure must come back as GMRF_E_INVALID.  Collected last so that it also runs
after every other GPU test in the same process.
"""
import numpy as np
import pytest

from paper_1702_05518_gb300 import gmrf as g
from paper_1702_05518_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1702_05518_gb300 import build

    build.build()


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def _graphs():
    r = wl.rng(9)
    rp, ci, _ = wl.delaunay_graph(20000, wl.rng(3))
    return {"grid8": wl.grid_graph(61, 45, eight=True), "er": wl.random_graph(3000, 0.003, r),
            "star": wl.star_graph(5000), "delaunay20k": (rp, ci),
            "isolated": wl.csr_from_edges(12, np.array([[0, 1], [1, 2], [7, 8]]))}


GRAPHS = _graphs()


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_noalloc_matches_colour_graph_twice(name):
    import torch

    rp, ci = GRAPHS[name]
    want, kw = g.color_graph(rp, ci, seed=17)
    rp_d, ci_d = _dev(rp), _dev(ci)
    for _ in range(2):
        col = torch.full((len(rp) - 1,), 12345, dtype=torch.int32, device="cuda")
        k = g.color_graph_noalloc(rp_d, ci_d, col, seed=17)
        assert k == kw
        assert np.array_equal(col.cpu().numpy(), want)


def test_noalloc_keeps_device_memory_unchanged():
    # the defining property: after a first call (which loads the library's device code), a call
    # takes no device memory
    import torch

    rp, ci = GRAPHS["delaunay20k"]
    rp_d, ci_d = _dev(rp), _dev(ci)
    col = torch.empty(len(rp) - 1, dtype=torch.int32, device="cuda")
    g.color_graph_noalloc(rp_d, ci_d, col, seed=3)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        g.color_graph_noalloc(rp_d, ci_d, col, seed=3)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_given_priorities():
    import torch

    rp, ci = GRAPHS["delaunay20k"]
    n = len(rp) - 1
    prio = (n - 1 - np.arange(n)).astype(np.uint32)
    want, kw = g.color_graph(rp, ci, priorities=prio)
    pr_d = torch.from_numpy(prio.view(np.int32)).cuda()
    for _ in range(2):
        col = torch.empty(n, dtype=torch.int32, device="cuda")
        assert g.color_graph_noalloc(_dev(rp), _dev(ci), col, priorities=pr_d) == kw
        assert np.array_equal(col.cpu().numpy(), want)


def test_noalloc_rejects_size_beyond_capacity():
    import torch

    n = 1 << 20
    rp, ci = wl.grid_graph(1024, 1024)
    col = torch.empty(n, dtype=torch.int32, device="cuda")
    assert g.color_graph_noalloc(_dev(rp), _dev(ci), col, seed=1) >= 2  # exactly at capacity
    rp1 = torch.zeros(n + 2, dtype=torch.int32, device="cuda")
    col1 = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(g.GmrfError, match="exceeds the static scratch") as e:
        g.color_graph_noalloc(rp1, torch.zeros(1, dtype=torch.int32, device="cuda")[:0], col1)
    assert e.value.status == g.E_INVALID


def test_noalloc_rejects_bad_structure():
    import torch

    rp, ci = wl.grid_graph(8, 9)
    n = len(rp) - 1
    col = torch.empty(n, dtype=torch.int32, device="cuda")
    bad_col = ci.copy()
    bad_col[5] = n  # one past the end: caught by the device check, never used as an index
    with pytest.raises(g.GmrfError, match="out of range"):
        g.color_graph_noalloc(_dev(rp), _dev(bad_col), col)
    loop = ci.copy()
    loop[rp[3]] = 3
    with pytest.raises(g.GmrfError, match="self-loop"):
        g.color_graph_noalloc(_dev(rp), _dev(loop), col)
    dec = rp.copy()
    dec[4] = dec[5] + 1
    with pytest.raises(g.GmrfError, match="non-decreasing|row_ptr"):
        g.color_graph_noalloc(_dev(dec), _dev(ci), col)
    with pytest.raises(g.GmrfError, match="row_ptr\\[n\\]"):
        g.color_graph_noalloc(_dev(rp), _dev(ci[:-1]), col)
    # a valid call right after the rejected ones still colours correctly
    want, kw = g.color_graph(rp, ci, seed=2)
    assert g.color_graph_noalloc(_dev(rp), _dev(ci), col, seed=2) == kw
    assert np.array_equal(col.cpu().numpy(), want)
