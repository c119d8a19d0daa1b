"""Pins of the oracle's coarse levels: the sparse Galerkin product equals the
literal dense P^T A P (Sec. 3), coarse operators of a pure Laplacian are again
Laplacians (A_H 1 = 0), aggregates are connected and disjoint (Sec. 2), the
lower-order term aggregates as P^T d, and the approximation property Eq. (wap)."""
import numpy as np
import pytest

import graphgen as gg
from helpers import dense_laplacian, prolongation, random_graph


def _connected(adj_rows, adj_col, members):
    ms = set(members)
    seen = {members[0]}
    stack = [members[0]]
    while stack:
        v = stack.pop()
        for j in adj_col[adj_rows[v]:adj_rows[v + 1]]:
            if j in ms and j not in seen:
                seen.add(int(j))
                stack.append(int(j))
    return len(seen) == len(ms)


CASES = [
    ("grid2d", lambda: gg.grid2d_5pt(20), 2),
    ("grid3d_d", lambda: gg.grid3d_7pt(8, 1.0), 3),
    ("rdiag", lambda: gg.grid2d_random_diag(16, 3), 3),
    ("rand_w", lambda: random_graph(150, 0.03, 4, wmax=5, d_frac=0.2), 2),
]


@pytest.mark.parametrize("name,make,passes", CASES)
def test_galerkin_equals_dense_triple_product(orc, name, make, passes):
    g = make()
    h = orc.Hierarchy(g, passes=passes, coarse_max=16)
    assert h.status == 0 and h.n_levels >= 2
    Ak = dense_laplacian(g)
    dk = np.zeros(g.n) if g.d is None else g.d.copy()
    for k in range(h.n_levels - 1):
        assert np.array_equal(h.level_dense(k), Ak)
        agg = h.level_agg(k)
        nH = h.level_n(k + 1)
        assert agg.min() == 0 and agg.max() == nH - 1 and np.unique(agg).size == nH
        P = prolongation(agg, nH)
        AH = P.T @ Ak @ P                                    # literal triple product
        assert np.array_equal(h.level_dense(k + 1), AH)      # integer weights: exact
        _, _, _, _, dlow = h.level_csr(k + 1)
        assert np.array_equal(dlow, P.T @ dk)
        if g.d is None:
            assert np.array_equal(AH @ np.ones(nH), np.zeros(nH))
        # aggregates are connected subgraphs of level k's graph, size <= 2^passes
        rp, col, _, _, _ = h.level_csr(k)
        order = np.argsort(agg, kind="stable")
        bounds = np.searchsorted(agg[order], np.arange(nH + 1))
        sizes = np.diff(bounds)
        assert sizes.max() <= 2 ** passes
        for I in range(nH):
            assert _connected(rp, col, order[bounds[I]:bounds[I + 1]].tolist())
        # composite map = composition of the per-pass maps
        comp = np.arange(h.level_n(k))
        for a in h.level_pass_aggs(k):
            comp = a[comp]
        assert np.array_equal(comp, agg)
        Ak, dk = AH, P.T @ dk


def test_approximation_property_wap(orc):
    """Eq. (wap): ||v - Qv||^2 <= c_p (Av, v), c_p = max_l 1/lambda_l with lambda_l
    the smallest positive eigenvalue of the Laplacian of aggregate l's subgraph."""
    g = gg.grid2d_5pt(12)
    h = orc.Hierarchy(g, passes=3, coarse_max=4)
    agg = h.level_agg(0)
    A = dense_laplacian(g)
    nH = agg.max() + 1
    cp = 0.0
    for l in range(nH):
        mem = np.nonzero(agg == l)[0]
        if mem.size < 2:
            continue
        W = -A[np.ix_(mem, mem)]
        np.fill_diagonal(W, 0)                              # edge weights inside aggregate l
        Al = np.diag(W.sum(axis=1)) - W                     # subgraph Laplacian A_l
        ev = np.linalg.eigvalsh(Al)
        assert ev[1] > 1e-12                                # connected subgraph
        cp = max(cp, 1.0 / ev[1])
    P = prolongation(agg, nH)
    Q = P @ np.diag(1.0 / P.sum(axis=0)) @ P.T              # Eq. (Q): aggregate means
    assert np.allclose(Q @ Q, Q) and np.allclose(Q, Q.T)
    assert 0 < cp < np.inf
    rng = np.random.default_rng(0)
    tight = 0.0
    for _ in range(50):
        v = rng.standard_normal(g.n)
        e = v - Q @ v
        assert e @ e <= cp * (v @ A @ v) * (1 + 1e-12)
        tight = max(tight, (e @ e) / (cp * (v @ A @ v)))
    assert tight > 0.01                                        # the bound is not vacuous
    assert np.allclose(P.T @ np.ones(g.n), np.bincount(agg))  # P^T 1 = aggregate sizes
    assert np.allclose(P @ np.ones(nH), 1.0)                   # P 1_H = 1
