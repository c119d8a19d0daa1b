"""Seeded synthetic inputs: graphs in CSR form and right-hand sides.

This module is the only code shared by the CUDA library's tests/benchmark and
the CPU oracle.  It holds no arithmetic of the solver: it only builds graphs
(vertex/edge structure, unit weights, lower-order terms) and random vectors.

Graphs stand in for the paper's workloads (Sec. 4): graph Laplacians of linear
finite elements for the Poisson problem on structured 2D/3D meshes, plus a
randomly triangulated 2D mesh and random geometric graphs for unstructured
cases, and Delaunay tetrahedralisations of perturbed 3D grids.  Every CSR
produced here is symmetric, has no self loops and has
strictly increasing column indices in each row.

Random numbers come from splitmix64 (S. Vigna's published finaliser of the
SplitMix64 generator) evaluated at ``seed XOR index``; a double in [0, 1) is
``(z >> 11) * 2**-53``.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """Vectorised splitmix64 finaliser on uint64 inputs (wrapping arithmetic)."""
    z = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1): u_k = (splitmix64(seed ^ (offset + k)) >> 11) * 2^-53."""
    idx = np.arange(offset, offset + n, dtype=np.uint64)
    z = splitmix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ idx)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, n: int) -> np.ndarray:
    """n doubles uniform on [-1, 1): 2u - 1."""
    return 2.0 * uniform01(seed, n) - 1.0


def rhs(n: int, seed: int, zero_mean: bool) -> np.ndarray:
    """Seeded uniform[-1,1] right-hand side; projected to zero mean (in fp64)
    when the operator is a pure graph Laplacian, whose range is 1-perp."""
    b = uniform_pm1(seed, n)
    if zero_mean:
        b = b - b.mean()
    return b


@dataclass
class Graph:
    """Undirected weighted graph in symmetric CSR form.

    rowptr: int64[n+1]; col: int32[nnz]; w: float64[nnz] (edge weights,
    each undirected edge stored twice); d: float64[n] lower-order terms or None.
    """

    n: int
    rowptr: np.ndarray
    col: np.ndarray
    w: np.ndarray
    d: Optional[np.ndarray]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    @property
    def n_edges(self) -> int:
        return self.nnz // 2


def _csr_from_masks(n: int, offsets, masks) -> tuple[np.ndarray, np.ndarray]:
    """Build CSR when each vertex v has candidate neighbours v + offsets[k]
    (offsets strictly increasing) present where masks[k][v] is True."""
    offs = np.asarray(offsets, dtype=np.int64)
    present = np.stack(masks, axis=1)  # n x K
    deg = present.sum(axis=1).astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=rowptr[1:])
    v = np.arange(n, dtype=np.int64)
    cand = v[:, None] + offs[None, :]
    col = cand[present].astype(np.int32)  # row-major order keeps rows sorted
    return rowptr, col


def grid2d_5pt(N: int) -> Graph:
    """N x N vertex grid, 5-point stencil graph, unit weights, no lower-order term.

    This is the graph of linear FE for Poisson on a uniform right-triangle mesh
    (the diagonal edges carry zero stiffness).  Vertex (i, j) -> i*N + j.
    """
    n = N * N
    v = np.arange(n, dtype=np.int64)
    i, j = v // N, v % N
    offsets = [-N, -1, 1, N]
    masks = [i > 0, j > 0, j < N - 1, i < N - 1]
    rowptr, col = _csr_from_masks(n, offsets, masks)
    return Graph(n, rowptr, col, np.ones(col.size), None, f"grid2d_5pt_{N}")


def grid3d_7pt(N: int, boundary_d: Optional[float] = 1.0) -> Graph:
    """N^3 vertex grid, 7-point stencil, unit weights.

    If boundary_d is not None, vertices on the boundary faces (some coordinate
    0 or N-1) carry the lower-order term d_i = boundary_d (Eq. (1)), all others 0.
    Vertex (k, i, j) -> (k*N + i)*N + j.
    """
    n = N * N * N
    v = np.arange(n, dtype=np.int64)
    j = v % N
    i = (v // N) % N
    k = v // (N * N)
    offsets = [-N * N, -N, -1, 1, N, N * N]
    masks = [k > 0, i > 0, j > 0, j < N - 1, i < N - 1, k < N - 1]
    rowptr, col = _csr_from_masks(n, offsets, masks)
    d = None
    if boundary_d is not None:
        bnd = (i == 0) | (i == N - 1) | (j == 0) | (j == N - 1) | (k == 0) | (k == N - 1)
        d = np.where(bnd, float(boundary_d), 0.0)
    return Graph(n, rowptr, col, np.ones(col.size), d, f"grid3d_7pt_{N}")


def square_orientation(N: int, seed: int) -> np.ndarray:
    """Orientation bit of each square (i, j), 0 <= i, j < N-1, of an N x N grid:
    bit 0 of splitmix64(seed ^ (i*N + j)).  0: diagonal (i,j)-(i+1,j+1);
    1: anti-diagonal (i+1,j)-(i,j+1).  Returned as an (N-1) x (N-1) uint8 array."""
    ii, jj = np.meshgrid(np.arange(N - 1, dtype=np.uint64), np.arange(N - 1, dtype=np.uint64), indexing="ij")
    z = splitmix64(np.uint64(seed) ^ (ii * np.uint64(N) + jj))
    return (z & np.uint64(1)).astype(np.uint8)


def grid2d_random_diag(N: int, seed: int) -> Graph:
    """N x N vertex grid where every square is split into two triangles along a
    seeded random diagonal: 5-point edges plus one diagonal per square, unit
    weights, pure graph Laplacian (no lower-order term)."""
    n = N * N
    o = square_orientation(N, seed)
    v = np.arange(n, dtype=np.int64)
    i, j = v // N, v % N

    def sq(ii, jj, valid):
        # orientation of square (ii, jj) where valid, else 255
        out = np.full(n, 255, dtype=np.uint8)
        out[valid] = o[ii[valid], jj[valid]]
        return out

    # candidate neighbours in increasing index order
    offsets = [-N - 1, -N, -N + 1, -1, 1, N - 1, N, N + 1]
    m_ul = sq(i - 1, j - 1, (i > 0) & (j > 0)) == 0          # (i-1,j-1): square (i-1,j-1), diag
    m_ur = sq(i - 1, j, (i > 0) & (j < N - 1)) == 1          # (i-1,j+1): square (i-1,j), anti-diag
    m_dl = sq(i, j - 1, (i < N - 1) & (j > 0)) == 1          # (i+1,j-1): square (i,j-1), anti-diag
    m_dr = sq(i, j, (i < N - 1) & (j < N - 1)) == 0          # (i+1,j+1): square (i,j), diag
    masks = [m_ul, i > 0, m_ur, j > 0, j < N - 1, m_dl, i < N - 1, m_dr]
    rowptr, col = _csr_from_masks(n, offsets, masks)
    return Graph(n, rowptr, col, np.ones(col.size), None, f"grid2d_rdiag_{N}_s{seed}")


def csr_from_edges(n: int, u: np.ndarray, v: np.ndarray, w: Optional[np.ndarray] = None,
                   d: Optional[np.ndarray] = None, name: str = "") -> Graph:
    """Symmetric CSR from an undirected edge list (u != v, no duplicates)."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    if w is None:
        w = np.ones(u.size)
    w = np.asarray(w, dtype=np.float64)
    rows = np.concatenate([u, v])
    cols = np.concatenate([v, u])
    ws = np.concatenate([w, w])
    order = np.argsort(rows * n + cols, kind="stable")
    rows, cols, ws = rows[order], cols[order], ws[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return Graph(n, rowptr, cols.astype(np.int32), ws, d, name)


def random_geometric(n: int, seed: int, mean_degree: float = 8.0) -> Graph:
    """Random geometric graph in the unit square, largest connected component.

    n points uniform in [0,1)^2 (x from seed, y from seed + 1); edge between
    points closer than r = sqrt(mean_degree / (pi n)).  Built with a cell list.
    The largest connected component is kept and its vertices relabelled in
    ascending original order; unit weights, no lower-order term.
    """
    x = uniform01(seed, n)
    y = uniform01(seed + 1, n)
    r = float(np.sqrt(mean_degree / (np.pi * n)))
    ncell = max(1, int(1.0 / r))
    cx = np.minimum((x * ncell).astype(np.int64), ncell - 1)
    cy = np.minimum((y * ncell).astype(np.int64), ncell - 1)
    cell = cx * ncell + cy
    order = np.argsort(cell, kind="stable")
    starts = np.searchsorted(cell[order], np.arange(ncell * ncell + 1))
    us, vs = [], []
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            ncx, ncy = cx + dx, cy + dy
            ok = (ncx >= 0) & (ncx < ncell) & (ncy >= 0) & (ncy < ncell)
            idx = np.nonzero(ok)[0]
            nc = ncx[idx] * ncell + ncy[idx]
            lo, hi = starts[nc], starts[nc + 1]
            cnt = hi - lo
            rep = np.repeat(idx, cnt)
            base = np.repeat(lo - np.cumsum(np.concatenate([[0], cnt[:-1]])), cnt)
            cand = order[base + np.arange(cnt.sum())]
            keep = (rep < cand) & ((x[rep] - x[cand]) ** 2 + (y[rep] - y[cand]) ** 2 < r * r)
            us.append(rep[keep])
            vs.append(cand[keep])
    u = np.concatenate(us)
    v = np.concatenate(vs)
    # largest connected component (ties: the component holding the smallest vertex)
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    adj = coo_matrix((np.ones(u.size), (u, v)), shape=(n, n)).tocsr()
    _, roots = connected_components(adj, directed=False)
    big = np.bincount(roots, minlength=n).argmax()
    keepv = roots == big
    newid = np.full(n, -1, dtype=np.int64)
    newid[keepv] = np.arange(int(keepv.sum()))
    ke = keepv[u] & keepv[v]
    return csr_from_edges(int(keepv.sum()), newid[u[ke]], newid[v[ke]], name=f"rgg_{n}_s{seed}")


def delaunay3d(N: int, seed: int) -> Graph:
    """Graph of an unstructured tetrahedral mesh of the unit cube, built as in
    the paper's unstructured test (Sec. 4): the N^3 vertices of a structured
    grid of spacing h = 1/(N-1) are each moved by a random vector of length
    h/2 (direction: the normalised vector (2u-1, 2u-1, 2u-1) with u from
    seed, seed + 1, seed + 2), then Delaunay-tetrahedralised (Qhull, through
    scipy.spatial).  The graph has the mesh's edges with unit weights and no
    lower-order term (the pure Laplacian of the mesh graph)."""
    from scipy.spatial import Delaunay

    n = N * N * N
    h = 1.0 / (N - 1)
    ax = np.linspace(0.0, 1.0, N)
    pts = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    dirs = np.stack([2.0 * uniform01(seed + c, n) - 1.0 for c in range(3)], -1)
    nrm = np.linalg.norm(dirs, axis=1, keepdims=True)
    nrm[nrm == 0.0] = 1.0
    pts = pts + dirs / nrm * (h / 2.0)
    tets = Delaunay(pts).simplices.astype(np.int64)
    e = np.concatenate([tets[:, [a, b]] for a in range(4) for b in range(a + 1, 4)])
    e.sort(axis=1)
    e = np.unique(e[:, 0] * n + e[:, 1])
    return csr_from_edges(n, e // n, e % n, name=f"delaunay3d_{N}_s{seed}")


# Named workloads (sizes and seeds of the benchmark configurations).
def workload(name: str) -> tuple[Graph, dict]:
    """Return (graph, solver parameters) for a named workload.

    grid2d_64     : 64x64 5-point Laplacian, pure, degree 3, 2 passes, seed 1
    grid3d_128    : 128^3 7-point, d=1 on boundary faces, degree 5, 3 passes, seed 2
    rdiag2d_2048  : 2048^2 random-diagonal triangulation, pure, degree 4, 3 passes,
                    matrix seed 3, RHS seed 1003, fp32 preconditioner
    grid3d_96x32  : 96^3 7-point, d=1 on boundary, 32 RHS seeds 4000..4031,
                    degree 5, 3 passes, fp32 preconditioner
    grid3d_128_neumann_mis : 128^3 7-point, pure (Neumann) Laplacian, degree 4,
                    aggregation by the independent set of the graph of A^4
                    (the setting of the paper's Table), RHS seed 2
    delaunay3d_64_mis : 64^3 unstructured tetrahedral mesh (perturbed grid +
                    Delaunay, seed 5), pure Laplacian of the mesh graph, degree
                    4, the same aggregation (the paper's unstructured column)
    """
    if name == "grid2d_64":
        g = grid2d_5pt(64)
        return g, dict(degree=3, passes=2, rhs_seeds=[1], precision=0)
    if name == "grid3d_128":
        g = grid3d_7pt(128, 1.0)
        return g, dict(degree=5, passes=3, rhs_seeds=[2], precision=0)
    if name == "rdiag2d_2048":
        g = grid2d_random_diag(2048, 3)
        return g, dict(degree=4, passes=3, rhs_seeds=[1003], precision=1)
    if name == "grid3d_128_neumann_mis":
        g = grid3d_7pt(128, None)
        return g, dict(degree=4, passes=1, rhs_seeds=[2], precision=0, aggregation=1)
    if name == "delaunay3d_64_mis":
        g = delaunay3d(64, 5)
        return g, dict(degree=4, passes=1, rhs_seeds=[5], precision=0, aggregation=1)
    if name == "grid3d_96x32":
        g = grid3d_7pt(96, 1.0)
        return g, dict(degree=5, passes=3, rhs_seeds=list(range(4000, 4032)), precision=1)
    raise KeyError(name)


def serve_graph_specs(count: int, seed: int = 5) -> list[tuple[str, int, int]]:
    """The serving workload's graphs as (kind, n, seed): target sizes
    log-uniform in [1e4, 1e6] (u from splitmix64(seed ^ index)); kinds cycle
    random geometric, random geometric, 2D 5-point grid, 3D 7-point grid (half
    random geometric graphs, a quarter each grid shape of the nearest size)."""
    u = uniform01(seed, count)
    sizes = np.exp(np.log(1e4) + u * np.log(100.0))
    kinds = ("rgg", "rgg", "grid2d", "grid3d")
    return [(kinds[i % 4], int(sizes[i]), 100 * seed + i) for i in range(count)]


def serve_graph(spec: tuple[str, int, int]) -> Graph:
    """Build one graph of serve_graph_specs (pure Laplacians, unit weights)."""
    kind, n, sd = spec
    if kind == "rgg":
        return random_geometric(n, sd)
    if kind == "grid2d":
        return grid2d_5pt(max(2, int(round(np.sqrt(n)))))
    return grid3d_7pt(max(2, int(round(n ** (1.0 / 3.0)))), None)


def is_pure_laplacian(g: Graph) -> bool:
    return g.d is None or not np.any(g.d)
