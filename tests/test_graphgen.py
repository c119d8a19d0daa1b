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
