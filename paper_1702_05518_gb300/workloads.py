"""Seeded synthetic inputs for the chromatic Gibbs sampler.

This module only generates data: observed fields y, true images, graphs (Delaunay
triangulations, small test graphs), initial states.  It holds none of the sampler's arithmetic,
and it is the one module both the CUDA path's callers and the oracle's tests draw inputs from.

The workloads stand in for the paper's experiments: the 2-D images of Sec. 3.1 (a smooth truth
plus Gaussian noise on a p x p lattice) and the irregular precinct graph of Sec. 3.2 (stood in
for by a Delaunay triangulation of uniform points, which is planar with mean degree near 6 like
an adjacency map of areal units).  Every generator takes an explicit seed and uses numpy's PCG64.
"""
from __future__ import annotations

import numpy as np

LATTICE2D_4, LATTICE2D_8, LATTICE3D_6, CSR = 0, 1, 2, 3


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


# --------------------------------------------------------------------------------------------
# Truth images
# --------------------------------------------------------------------------------------------
def block_image(H: int, W: int) -> np.ndarray:
    """Piecewise-constant 4-level image: level(i, j) = (floor(4i/H) + floor(4j/W)) mod 4."""
    i = np.arange(H)[:, None]
    j = np.arange(W)[None, :]
    return (((4 * i) // H + (4 * j) // W) % 4).astype(np.float64)


def gaussian_bumps(H: int, W: int, nbumps: int, g: np.random.Generator) -> np.ndarray:
    """Sum of `nbumps` isotropic Gaussian bumps, amplitude U(0,3), width U(5,50) px, centres
    uniform over the grid."""
    amp = g.uniform(0.0, 3.0, nbumps)
    width = g.uniform(5.0, 50.0, nbumps)
    ci = g.uniform(0.0, H, nbumps)
    cj = g.uniform(0.0, W, nbumps)
    ii = np.arange(H, dtype=np.float64)[:, None]
    jj = np.arange(W, dtype=np.float64)[None, :]
    img = np.zeros((H, W))
    for b in range(nbumps):
        img += amp[b] * np.exp(-((ii - ci[b]) ** 2 + (jj - cj[b]) ** 2) / (2.0 * width[b] ** 2))
    return img


def paper_image(p: int) -> np.ndarray:
    """The true image of the paper's simulation (Sec. 3.1): a rescaled bivariate normal density
    5 exp(-|v|^2 / 2) / pi over pixel centres evenly spaced on [-3, 3]^2."""
    v = np.linspace(-3.0, 3.0, p)
    return 5.0 * np.exp(-(v[:, None] ** 2 + v[None, :] ** 2) / 2.0) / np.pi


def ellipsoids(L: int, H: int, W: int, nell: int, g: np.random.Generator) -> np.ndarray:
    """Sum of `nell` axis-aligned solid ellipsoids, amplitude U(0.5, 2), centres uniform over
    the volume, semi-axes U(4, 32) voxels per axis."""
    amp = g.uniform(0.5, 2.0, nell)
    cen = g.uniform(0.0, 1.0, (nell, 3)) * np.array([L, H, W])
    ax = g.uniform(4.0, 32.0, (nell, 3))
    vol = np.zeros((L, H, W), np.float64)
    for e in range(nell):
        lo = np.maximum(np.floor(cen[e] - ax[e]).astype(int), 0)
        hi = np.minimum(np.ceil(cen[e] + ax[e]).astype(int) + 1, [L, H, W])
        if np.any(hi <= lo):
            continue
        l = np.arange(lo[0], hi[0])[:, None, None]
        i = np.arange(lo[1], hi[1])[None, :, None]
        j = np.arange(lo[2], hi[2])[None, None, :]
        inside = (((l - cen[e, 0]) / ax[e, 0]) ** 2 + ((i - cen[e, 1]) / ax[e, 1]) ** 2
                  + ((j - cen[e, 2]) / ax[e, 2]) ** 2) <= 1.0
        vol[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] += amp[e] * inside
    return vol


# --------------------------------------------------------------------------------------------
# Graphs (symmetric CSR, sorted rows, no self-loops, no duplicates)
# --------------------------------------------------------------------------------------------
def csr_from_edges(n: int, edges: np.ndarray):
    """Symmetric CSR from an [m, 2] array of undirected edges (duplicates removed)."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    e = e[e[:, 0] != e[:, 1]]
    both = np.concatenate([e, e[:, ::-1]], axis=0)
    key = np.unique(both[:, 0] * np.int64(n) + both[:, 1]) if len(both) else np.zeros(0, np.int64)
    rows = (key // n).astype(np.int64)
    cols = (key % n).astype(np.int32)
    row_ptr = np.zeros(n + 1, np.int32)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    return row_ptr, cols


def delaunay_graph(npts: int, g: np.random.Generator):
    """Delaunay triangulation of `npts` uniform points in the unit square -> (row_ptr, col_idx,
    points [npts, 2]).  Planar, mean degree just under 6."""
    from scipy.spatial import Delaunay

    pts = g.uniform(0.0, 1.0, (npts, 2))
    tri = Delaunay(pts)
    s = tri.simplices
    edges = np.concatenate([s[:, [0, 1]], s[:, [1, 2]], s[:, [0, 2]]], axis=0)
    rp, ci = csr_from_edges(npts, edges)
    return rp, ci, pts


def path_graph(n: int):
    return csr_from_edges(n, np.stack([np.arange(n - 1), np.arange(1, n)], axis=1))


def cycle_graph(n: int):
    return csr_from_edges(n, np.stack([np.arange(n), (np.arange(n) + 1) % n], axis=1))


def k4_minus_edge():
    """Complete graph on 4 vertices with the edge {0, 3} removed (needs 3 colours)."""
    return csr_from_edges(4, np.array([[0, 1], [0, 2], [1, 2], [1, 3], [2, 3]]))


def grid_graph(H: int, W: int, eight: bool = False):
    """Free-boundary H x W grid as an explicit CSR graph (row-major site order)."""
    idx = np.arange(H * W).reshape(H, W)
    e = [np.stack([idx[:, :-1].ravel(), idx[:, 1:].ravel()], 1),
         np.stack([idx[:-1, :].ravel(), idx[1:, :].ravel()], 1)]
    if eight:
        e.append(np.stack([idx[:-1, :-1].ravel(), idx[1:, 1:].ravel()], 1))
        e.append(np.stack([idx[:-1, 1:].ravel(), idx[1:, :-1].ravel()], 1))
    return csr_from_edges(H * W, np.concatenate(e, 0))


def random_graph(n: int, p: float, g: np.random.Generator):
    """Erdos-Renyi G(n, p) as CSR (for colouring and edge-case tests)."""
    iu = np.triu_indices(n, 1)
    keep = g.uniform(size=len(iu[0])) < p
    return csr_from_edges(n, np.stack([iu[0][keep], iu[1][keep]], 1))


def star_graph(n: int):
    """Vertex 0 joined to 1..n-1: one vertex of high degree (degree n-1)."""
    return csr_from_edges(n, np.stack([np.zeros(n - 1, np.int64), np.arange(1, n)], 1))


def prior_draw(row_ptr, col_idx, tau: float, rho: float, g: np.random.Generator):
    """x ~ N(0, (tau (D - rho W))^-1) for a proper CAR (rho < 1), unit weights.

    With B the signed incidence matrix (D - W = B B^T), tau (D - rho W) = A A^T for
    A = sqrt(tau) [sqrt((1 - rho) D), sqrt(rho) B], so x = (tau (D - rho W))^-1 A z has the
    required covariance; one sparse direct solve."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    rp = np.asarray(row_ptr, np.int64)
    ci = np.asarray(col_idx, np.int64)
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    Wm = sp.csr_matrix((np.ones(len(ci)), (rows, ci)), shape=(n, n))
    d = np.asarray(Wm.sum(axis=1)).ravel()
    Q = (tau * (sp.diags(d) - rho * Wm)).tocsc()
    up = rows < ci
    eu, ev = rows[up], ci[up]
    z1 = g.standard_normal(n)
    z2 = g.standard_normal(len(eu))
    bz = np.sqrt((1.0 - rho) * d) * z1
    np.add.at(bz, eu, np.sqrt(rho) * z2)
    np.add.at(bz, ev, -np.sqrt(rho) * z2)
    return spla.spsolve(Q, np.sqrt(tau) * bz)


# --------------------------------------------------------------------------------------------
# The five workloads (a field = dict(kind, dims, n, y, truth, [row_ptr, col_idx, points]))
# --------------------------------------------------------------------------------------------
def lattice_field(kind, dims, truth, noise_sd, g):
    y = truth + noise_sd * g.standard_normal(truth.shape)
    return {"kind": kind, "dims": tuple(int(d) for d in dims), "n": int(truth.size),
            "y": y.ravel().astype(np.float64), "truth": truth.ravel()}


def image_64_block(seed: int = 0):
    """64 x 64 first-order (4-neighbour) ICAR, checkerboard; 4-level block image + N(0, 0.5^2)."""
    g = rng(seed)
    return [lattice_field(LATTICE2D_4, (64, 64), block_image(64, 64), 0.5, g)]


def image_1024_bumps(seed: int = 2, side: int = 1024):
    """side x side second-order (8-neighbour) ICAR, 2x2 colouring; 20 Gaussian bumps + N(0,1)."""
    g = rng(seed)
    return [lattice_field(LATTICE2D_8, (side, side), gaussian_bumps(side, side, 20, g), 1.0, g)]


def delaunay_pcar(seed: int = 3, npts: int = 16384, tau_true: float = 4.0, rho: float = 0.95,
                  noise_sd: float = 0.3):
    """Delaunay graph of `npts` uniform points, proper CAR; x_true from the prior at tau_true,
    y = x_true + N(0, noise_sd^2)."""
    g = rng(seed)
    rp, ci, pts = delaunay_graph(npts, g)
    xt = prior_draw(rp, ci, tau_true, rho, g)
    y = xt + noise_sd * g.standard_normal(npts)
    return [{"kind": CSR, "dims": (npts, 0, 0), "n": npts, "y": y, "truth": xt,
             "row_ptr": rp, "col_idx": ci, "points": pts}]


def binomial_delaunay(seed: int = 7, npts: int = 14926, tau_true: float = 2.0, rho: float = 0.995,
                      beta0_true: float = 0.4, trials_range=(1, 64), missing: float = 0.022):
    """Stand-in for the precinct vote counts of Sec. 3.2 (the election data are not available):
    a Delaunay graph of `npts` uniform points, x_true from the proper CAR prior at tau_true,
    success probability logistic(beta0_true + x_true), trials log-uniform in trials_range
    (integers), a fraction `missing` of sites without data (0 trials), successes binomial."""
    g = rng(seed)
    rp, ci, pts = delaunay_graph(npts, g)
    xt = prior_draw(rp, ci, tau_true, rho, g)
    lo, hi = np.log(trials_range[0]), np.log(trials_range[1] + 1)
    m = np.floor(np.exp(g.uniform(lo, hi, npts))).astype(np.int32)
    m[g.uniform(size=npts) < missing] = 0
    p = 1.0 / (1.0 + np.exp(-(beta0_true + xt)))
    y = g.binomial(m, p).astype(np.float64)
    return [{"kind": CSR, "dims": (npts, 0, 0), "n": npts, "y": y, "trials": m, "truth": xt,
             "row_ptr": rp, "col_idx": ci, "points": pts}]


def batched_uneven(seed: int = 4, nlat: int = 224, ngraph: int = 32, side_range=(32, 512),
                   n_range=(1000, 50000)):
    """Many independent fields of uneven sizes: `nlat` 4-neighbour lattices with sides
    log-uniform in side_range and `ngraph` Delaunay graphs with n log-uniform in n_range; each
    y = 4-level block image + N(0, 0.5^2)."""
    g = rng(seed)
    fields = []
    for _ in range(nlat):
        s = int(round(np.exp(g.uniform(np.log(side_range[0]), np.log(side_range[1])))))
        fields.append(lattice_field(LATTICE2D_4, (s, s), block_image(s, s), 0.5, g))
    for _ in range(ngraph):
        m = int(round(np.exp(g.uniform(np.log(n_range[0]), np.log(n_range[1])))))
        rp, ci, pts = delaunay_graph(m, g)
        truth = ((np.floor(4 * pts[:, 0]) + np.floor(4 * pts[:, 1])) % 4).astype(np.float64)
        y = truth + 0.5 * g.standard_normal(m)
        fields.append({"kind": CSR, "dims": (m, 0, 0), "n": m, "y": y, "truth": truth,
                       "row_ptr": rp, "col_idx": ci, "points": pts})
    return fields


def volume_ellipsoids(seed: int = 5, side: int = 256):
    """side^3 first-order (6-neighbour) ICAR, parity colouring; 50 ellipsoids + N(0, 1)."""
    g = rng(seed)
    truth = ellipsoids(side, side, side, 50, g)
    y = truth + g.standard_normal(truth.shape, dtype=np.float64)
    return [{"kind": LATTICE3D_6, "dims": (side, side, side), "n": int(truth.size),
             "y": y.ravel(), "truth": truth.ravel()}]


def small_lattice(kind, dims, seed: int, noise_sd: float = 0.5):
    """A small lattice field with a block-image truth (2-D) or a random truth (3-D)."""
    g = rng(seed)
    if kind == LATTICE3D_6:
        truth = g.uniform(0.0, 3.0, dims)
    else:
        truth = block_image(dims[0], dims[1])
    return lattice_field(kind, dims, truth, noise_sd, g)


def graph_field(row_ptr, col_idx, seed: int, noise_sd: float = 0.5):
    """A CSR field over a given graph with a random truth."""
    g = rng(seed)
    n = len(row_ptr) - 1
    truth = g.uniform(0.0, 3.0, n)
    return {"kind": CSR, "dims": (n, 0, 0), "n": n, "y": truth + noise_sd * g.standard_normal(n),
            "truth": truth, "row_ptr": np.asarray(row_ptr, np.int32),
            "col_idx": np.asarray(col_idx, np.int32)}
