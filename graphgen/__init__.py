"""Seeded synthetic graph and right-hand-side generators.

This module only builds inputs: symmetric weighted adjacency structures (no diagonal, no
Laplacian arithmetic of the solver) and the right-hand sides the paper's experiments use
(Section 4: ``b = L x_true`` with ``x_true`` standard normal, projected to zero mean).
Both the CPU oracle and the CUDA library consume what it returns; it imports neither.

Every graph is returned as a ``Graph``: ``n`` nodes, CSR arrays ``rp`` (int64, n+1),
``ci`` (int32, column ids sorted ascending per row, no self loops) and ``w`` (float64,
positive edge weights, symmetric: w[u->v] == w[v->u]).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Graph:
    n: int
    rp: np.ndarray   # int64 [n+1]
    ci: np.ndarray   # int32 [nnz]
    w: np.ndarray    # float64 [nnz]
    name: str = ""

    @property
    def nnz_off(self) -> int:
        return int(self.rp[-1])

    @property
    def m(self) -> int:
        """Number of undirected edges."""
        return int(self.rp[-1]) // 2

    @property
    def nnz_L(self) -> int:
        """nnz of the Laplacian, diagonal included: n + 2m."""
        return self.n + int(self.rp[-1])


def from_edges(n: int, u, v, w, name: str = "") -> Graph:
    """Build a symmetric CSR adjacency from an undirected edge list (u != v, no duplicates
    after ordering the pair; duplicates are merged by summing weights)."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    keep = u != v
    u, v, w = u[keep], v[keep], w[keep]
    a = np.minimum(u, v)
    b = np.maximum(u, v)
    key = a * n + b
    order = np.argsort(key, kind="stable")
    key, w = key[order], w[order]
    uniq, start = np.unique(key, return_index=True)
    wsum = np.add.reduceat(w, start) if len(key) else w
    a = uniq // n
    b = uniq % n
    rows = np.concatenate([a, b])
    cols = np.concatenate([b, a])
    ws = np.concatenate([wsum, wsum])
    order = np.lexsort((cols, rows))
    rows, cols, ws = rows[order], cols[order], ws[order]
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, rows + 1, 1)
    rp = np.cumsum(rp)
    return Graph(n, rp, cols.astype(np.int32), ws.astype(np.float64), name)


def grid2d(nx: int, ny: int, wx: float = 1.0, wy: float = 1.0) -> Graph:
    """5-point grid; node id = i + nx*j; x-edges weight wx, y-edges weight wy."""
    idx = np.arange(nx * ny, dtype=np.int64).reshape(ny, nx)
    ux = idx[:, :-1].ravel(); vx = idx[:, 1:].ravel()
    uy = idx[:-1, :].ravel(); vy = idx[1:, :].ravel()
    u = np.concatenate([ux, uy]); v = np.concatenate([vx, vy])
    w = np.concatenate([np.full(ux.size, wx), np.full(uy.size, wy)])
    name = f"grid2d_{nx}x{ny}" + ("" if wx == wy == 1.0 else f"_wx{wx:g}_wy{wy:g}")
    return from_edges(nx * ny, u, v, w, name)


def grid3d(nx: int, ny: int, nz: int, weights: str = "unit", seed: int = 1,
           lo: float = 1e-3, hi: float = 1e3) -> Graph:
    """7-point grid; ``weights='loguniform'`` draws i.i.d. w = 10^U(log10 lo, log10 hi)."""
    idx = np.arange(nx * ny * nz, dtype=np.int64).reshape(nz, ny, nx)
    pairs = [(idx[:, :, :-1], idx[:, :, 1:]), (idx[:, :-1, :], idx[:, 1:, :]),
             (idx[:-1, :, :], idx[1:, :, :])]
    u = np.concatenate([p[0].ravel() for p in pairs])
    v = np.concatenate([p[1].ravel() for p in pairs])
    if weights == "unit":
        w = np.ones(u.size)
    elif weights == "loguniform":
        rng = np.random.default_rng(seed)
        w = 10.0 ** rng.uniform(math.log10(lo), math.log10(hi), size=u.size)
    else:
        raise ValueError(weights)
    return from_edges(nx * ny * nz, u, v, w, f"grid3d_{nx}x{ny}x{nz}_{weights}")


def aniso_patch(N: int, patch: int, eps: float) -> Graph:
    """Isotropic N x N grid with an anisotropic patch x patch block in the centre whose
    y-edges have weight eps (the locally-anisotropic graphs of the paper's Table 2)."""
    idx = np.arange(N * N, dtype=np.int64).reshape(N, N)
    lo = (N - patch) // 2
    ux = idx[:, :-1].ravel(); vx = idx[:, 1:].ravel()
    uy = idx[:-1, :].ravel(); vy = idx[1:, :].ravel()
    jy = (np.arange(N * N) // N).reshape(N, N)[:-1, :].ravel()
    iy = (np.arange(N * N) % N).reshape(N, N)[:-1, :].ravel()
    inpatch = (jy >= lo) & (jy < lo + patch - 1) & (iy >= lo) & (iy < lo + patch)
    wy = np.where(inpatch, eps, 1.0)
    return from_edges(N * N, np.concatenate([ux, uy]), np.concatenate([vx, vy]),
                      np.concatenate([np.ones(ux.size), wy]), f"patch{N}_{patch}_{eps:g}")


def grid2d_random(nx: int, ny: int, seed: int, wlo: float = 0.5, whi: float = 1.5) -> Graph:
    """5-point grid with i.i.d. weights U(wlo, whi]."""
    g = grid2d(nx, ny)
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(g.n), np.diff(g.rp))
    lo = np.minimum(rows, g.ci)
    hi = np.maximum(rows, g.ci)
    keep = rows < g.ci
    w = whi - (whi - wlo) * rng.random(int(keep.sum()))
    return from_edges(g.n, lo[keep], hi[keep], w, f"grid2d_{nx}x{ny}_rand")


def grid_with_hubs(nx: int, ny: int, hubs: int, deg: int, seed: int = 1) -> Graph:
    """A 2D 5-point grid (weights U(0.5, 1.5]) plus `hubs` extra nodes, each joined to `deg`
    distinct random grid nodes (weights U(0.5, 1.5]) and to the previous hub: a mesh with a
    few rows far longer than the rest, as power-law graphs have."""
    rng = np.random.default_rng(seed)
    g0 = grid2d_random(nx, ny, seed)
    ng = nx * ny
    n = ng + hubs
    r = np.repeat(np.arange(ng), np.diff(g0.rp))
    m = r < g0.ci
    us, vs, ws = [r[m]], [g0.ci[m].astype(np.int64)], [g0.w[m]]
    for h in range(hubs):
        nb = rng.choice(ng, size=deg, replace=False)
        us.append(np.full(deg, ng + h))
        vs.append(nb)
        ws.append(rng.uniform(0.5, 1.5, deg))
        if h:
            us.append(np.array([ng + h]))
            vs.append(np.array([ng + h - 1]))
            ws.append(np.array([1.0]))
    return from_edges(n, np.concatenate(us), np.concatenate(vs), np.concatenate(ws),
                      f"grid_hubs{nx}x{ny}_{hubs}x{deg}")


def path(n: int, w=None) -> Graph:
    u = np.arange(n - 1); v = u + 1
    w = np.ones(n - 1) if w is None else np.asarray(w, dtype=np.float64)
    return from_edges(n, u, v, w, f"path{n}")


def cycle(n: int, w=None) -> Graph:
    u = np.arange(n); v = (u + 1) % n
    w = np.ones(n) if w is None else np.asarray(w, dtype=np.float64)
    return from_edges(n, u, v, w, f"cycle{n}")


def star(n: int, w=None) -> Graph:
    """Hub 0 joined to leaves 1..n-1."""
    v = np.arange(1, n); u = np.zeros(n - 1, dtype=np.int64)
    w = np.ones(n - 1) if w is None else np.asarray(w, dtype=np.float64)
    return from_edges(n, u, v, w, f"star{n}")


def random_connected(n: int, extra: int, seed: int, wlo: float = 0.5, whi: float = 1.5) -> Graph:
    """Random spanning tree plus ``extra`` random edges; weights U(wlo, whi]."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    parent = np.array([perm[rng.integers(0, i)] for i in range(1, n)], dtype=np.int64)
    u = np.concatenate([perm[1:], rng.integers(0, n, extra)])
    v = np.concatenate([parent, rng.integers(0, n, extra)])
    w = whi - (whi - wlo) * rng.random(u.size)
    return from_edges(n, u, v, w, f"rand{n}_{extra}_s{seed}")


def largest_cc(g: Graph) -> Graph:
    """Restrict to the largest connected component (node ids renumbered in order)."""
    import scipy.sparse as sp
    import scipy.sparse.csgraph as csg
    A = sp.csr_matrix((g.w, g.ci, g.rp), shape=(g.n, g.n))
    ncomp, lab = csg.connected_components(A, directed=False)
    if ncomp == 1:
        return g
    big = np.bincount(lab).argmax()
    keep = np.flatnonzero(lab == big)
    sub = A[keep][:, keep].tocsr()
    sub.sort_indices()
    return Graph(len(keep), sub.indptr.astype(np.int64), sub.indices.astype(np.int32),
                 sub.data.astype(np.float64), g.name + "_lcc")


def chung_lu(n: int, exponent: float = 2.1, mean_deg: float = 16.0, seed: int = 1,
             wlo: float = 0.5, whi: float = 1.5) -> Graph:
    """Chung-Lu power-law graph: expected degrees from a Pareto density with the given
    exponent, scaled to the requested mean and capped at sqrt(sum of degrees). Edges are
    sampled as Poisson(S/2) endpoint pairs drawn proportionally to the expected degrees,
    with self loops and duplicates removed (an O(n+m) Chung-Lu sampler). Largest connected
    component only; weights U(wlo, whi]."""
    rng = np.random.default_rng(seed)
    a = exponent - 1.0
    d = (1.0 - rng.random(n)) ** (-1.0 / a)          # Pareto(x_min = 1)
    d *= mean_deg / d.mean()
    cap = math.sqrt(d.sum())
    d = np.minimum(d, cap)
    d *= mean_deg / d.mean()
    S = d.sum()
    m = rng.poisson(S / 2.0)
    p = d / S
    u = rng.choice(n, size=m, p=p)
    v = rng.choice(n, size=m, p=p)
    w = whi - (whi - wlo) * rng.random(m)
    g = from_edges(n, u, v, w, f"chunglu{n}")
    return largest_cc(g)


def rgg(n: int, mean_deg: float = 10.0, seed: int = 1, wlo: float = 0.5, whi: float = 1.5) -> Graph:
    """Random geometric graph in the unit square, radius r = sqrt(mean_deg / (pi n));
    largest connected component."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    r = math.sqrt(mean_deg / (math.pi * n))
    pairs = cKDTree(pts).query_pairs(r, output_type="ndarray")
    w = whi - (whi - wlo) * rng.random(len(pairs))
    g = from_edges(n, pairs[:, 0], pairs[:, 1], w, f"rgg{n}")
    return largest_cc(g)


def barabasi_albert(n: int, k: int = 4, seed: int = 1, wlo: float = 0.5, whi: float = 1.5) -> Graph:
    """Barabasi-Albert preferential attachment: each new node attaches k edges to existing
    nodes chosen proportionally to degree (sampled from the endpoint list)."""
    rng = np.random.default_rng(seed)
    m0 = k + 1
    us = []; vs = []
    for i in range(m0):
        for j in range(i + 1, m0):
            us.append(i); vs.append(j)
    ends = np.empty(2 * (len(us) + k * (n - m0)), dtype=np.int64)
    ne = 0
    for a, b in zip(us, vs):
        ends[ne] = a; ends[ne + 1] = b; ne += 2
    U = np.empty(k * (n - m0), dtype=np.int64); V = np.empty_like(U)
    t = 0
    for x in range(m0, n):
        picks = ends[rng.integers(0, ne, size=k)]
        for p in picks:
            U[t] = x; V[t] = p; t += 1
        for p in picks:
            ends[ne] = x; ends[ne + 1] = p; ne += 2
    u = np.concatenate([np.array(us), U]); v = np.concatenate([np.array(vs), V])
    w = whi - (whi - wlo) * rng.random(u.size)
    return from_edges(n, u, v, w, f"ba{n}_{k}")


def laplacian_apply(g: Graph, x: np.ndarray) -> np.ndarray:
    """(L x)_u = sum_v w_uv (x_u - x_v): the definition of L = D - W (Section 1, Eq. 1)."""
    import scipy.sparse as sp
    A = sp.csr_matrix((g.w, g.ci, g.rp), shape=(g.n, g.n))
    deg = np.asarray(A.sum(axis=1)).ravel()
    X = x if x.ndim == 2 else x[:, None]
    out = deg[:, None] * X - A @ X
    return out if x.ndim == 2 else out[:, 0]


def rhs(g: Graph, seed: int = 2, k: int = 1) -> np.ndarray:
    """b = L x_true with x_true ~ N(0,1) (numpy PCG64 seeded), x_true projected to zero mean,
    and b projected to zero mean (Section 4). Shape (n,) for k == 1, else (n, k)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((g.n, k))
    x -= x.mean(axis=0, keepdims=True)
    b = laplacian_apply(g, x)
    b -= b.mean(axis=0, keepdims=True)
    return b[:, 0].copy() if k == 1 else np.ascontiguousarray(b)


def config_graph(name: str) -> Graph:
    """The named synthetic workloads."""
    if name == "grid64":
        return grid2d(64, 64)
    if name == "aniso1024":
        return grid2d(1024, 1024, 1.0, 1e-3)
    if name == "grid3d192_hetero":
        return grid3d(192, 192, 192, "loguniform", seed=1)
    if name == "chunglu4m":
        return chung_lu(4_000_000, 2.1, 16.0, seed=1)
    raise KeyError(name)
