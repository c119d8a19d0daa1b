"""Checks of the seeded input generators (graphgen): structure and
determinism of the graphs that stand in for the paper's meshes (Sec. 4)."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

import graphgen as gg


def as_matrix(g):
    return sp.csr_matrix((g.w, g.col, g.rowptr), shape=(g.n, g.n))


@pytest.mark.parametrize("N", [6, 10])
def test_delaunay3d_mesh_graph(N):
    g = gg.delaunay3d(N, 5)
    A = as_matrix(g)
    assert g.n == N ** 3 and g.d is None
    assert (A != A.T).nnz == 0 and A.diagonal().sum() == 0         # symmetric, no loops
    assert np.all(np.diff(g.rowptr) > 0)
    for i in range(g.n):                                           # strictly increasing columns
        c = g.col[g.rowptr[i]:g.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    assert connected_components(A, directed=False)[0] == 1
    # a tetrahedral mesh of a perturbed grid: mean degree ~14-15 (Euler), each
    # grid neighbour of the structured mesh is typically still an edge
    mean = g.col.size / g.n
    assert 11.0 < mean < 17.0
    assert np.all(g.w == 1.0)


def test_delaunay3d_is_deterministic():
    a, b = gg.delaunay3d(8, 3), gg.delaunay3d(8, 3)
    assert np.array_equal(a.rowptr, b.rowptr) and np.array_equal(a.col, b.col)
    c = gg.delaunay3d(8, 4)
    assert not (np.array_equal(a.rowptr, c.rowptr) and np.array_equal(a.col, c.col))


@pytest.mark.parametrize("name,n,edges,nnz_diag,boundary,nrhs", [
    ("grid2d_64", 4096, 8064, 20224, 0, 1),
    ("grid3d_128", 2097152, 6242304, 14581760, 96776, 1),
    ("grid3d_96x32", 884736, 2626560, 6137856, 54152, 32),
    ("rdiag2d_2048", 4194304, 12574721, 29343746, 0, 1),
])
def test_workload_sizes(name, n, edges, nnz_diag, boundary, nrhs):
    """The synthetic workloads have the sizes of the benchmark configurations:
    vertices, undirected edges, stored entries with the diagonal, vertices
    carrying a lower-order term (the boundary faces), right-hand sides."""
    g, p = gg.workload(name)
    assert g.n == n and g.col.size == 2 * edges and g.col.size + g.n == nnz_diag
    assert (0 if g.d is None else int((g.d > 0).sum())) == boundary
    assert len(p["rhs_seeds"]) == nrhs


@pytest.mark.parametrize("n,seed", [(20000, 61), (100000, 3)])
def test_random_geometric_graph(n, seed):
    """Random geometric graphs in the unit square: the radius gives mean degree
    8; the largest component is kept (over 99% of the points), so the graph is
    connected, symmetric and a pure Laplacian."""
    g = gg.random_geometric(n, seed)
    A = sp.csr_matrix((np.ones(g.col.size), g.col, g.rowptr), shape=(g.n, g.n))
    assert 0.99 * n <= g.n <= n
    assert abs(g.col.size / g.n - 8.0) < 0.2
    assert connected_components(A, directed=False)[0] == 1
    assert (A != A.T).nnz == 0 and g.d is None
    assert np.all(np.diff(g.rowptr) > 0)
