"""Pins of the oracle's handshake matching (Sec. 2: a matching is a set of
non-incident edges, each matched edge a two-vertex aggregate) and of the
coarse numbering.  The handshake result is checked against a brute-force
sequential greedy matching by decreasing edge key: with a strict total order
on edges the locally-dominant handshake rule selects exactly the greedy set."""
import numpy as np
import pytest

import graphgen as gg
from helpers import random_graph

MASK = (1 << 64) - 1


def sm64(x):
    z = (x + 0x9E3779B97F4A7C15) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def greedy_matching(g, salt):
    edges = []
    for i in range(g.n):
        for p in range(g.rowptr[i], g.rowptr[i + 1]):
            j = int(g.col[p])
            if i < j:
                edges.append((g.w[p], sm64(salt ^ ((i << 32) | j)), i, j))
    edges.sort(reverse=True)
    mate = -np.ones(g.n, dtype=np.int64)
    for _, _, i, j in edges:
        if mate[i] < 0 and mate[j] < 0:
            mate[i], mate[j] = j, i
    return mate


def test_splitmix64_matches_generator_module():
    xs = np.array([0, 1, 2, 12345, (7 << 32) | 9], dtype=np.uint64)
    ref = gg.splitmix64(xs)
    assert [sm64(int(x)) for x in xs] == [int(v) for v in ref]


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("wmax", [1, 3])
def test_handshake_equals_greedy(orc, seed, wmax):
    g = random_graph(70, 0.07, seed=seed, wmax=wmax)
    salt = 1234567 * seed
    mate, agg, nH, rounds = orc.match(g.rowptr, g.col, g.w, salt)
    assert np.array_equal(mate, greedy_matching(g, salt))
    assert rounds >= 1


@pytest.mark.parametrize("make", [lambda: gg.grid2d_5pt(17), lambda: gg.grid3d_7pt(6, None),
                                  lambda: gg.random_geometric(500, 5), lambda: random_graph(90, 0.05, 9, wmax=4)])
def test_matching_is_maximal_and_numbered_by_representatives(orc, make):
    g = make()
    mate, agg, nH, _ = orc.match(g.rowptr, g.col, g.w, 99)
    n = g.n
    rows = np.repeat(np.arange(n), np.diff(g.rowptr))
    adj = set(zip(rows.tolist(), g.col.tolist()))
    for i in range(n):
        if mate[i] >= 0:
            assert mate[mate[i]] == i and (i, int(mate[i])) in adj
    # maximal: no edge with both ends unmatched
    assert not np.any((mate[rows] < 0) & (mate[g.col] < 0))
    # coarse ids: rank of the representative (unmatched, or smaller end of its pair)
    rep = (mate < 0) | (np.arange(n) < mate)
    rank = np.cumsum(rep) - 1
    owner = np.where(rep, np.arange(n), np.minimum(np.arange(n), mate))
    assert np.array_equal(agg, rank[owner])
    assert nH == rep.sum()
    assert np.all(np.bincount(agg, minlength=nH) <= 2) and np.all(np.bincount(agg) >= 1)


def numbered_by_representatives(mate):
    n = mate.size
    rep = (mate < 0) | (np.arange(n) < mate)
    rank = np.cumsum(rep) - 1
    owner = np.where(rep, np.arange(n), np.minimum(np.arange(n), mate))
    return rank[owner]


@pytest.mark.parametrize("make,passes", [
    (lambda: gg.grid2d_5pt(16), 3),
    (lambda: gg.grid3d_7pt(6, 1.0), 3),
    (lambda: random_graph(160, 0.03, 2, wmax=4, d_frac=0.1), 2),
])
def test_each_pass_is_the_greedy_matching_of_the_intermediate_graph(orc, make, passes):
    """Sec. 2 repeats pairwise matching on the graph of the previous pass's
    Galerkin operator.  Built here independently: B_0 = A_k from the graph and
    the composite maps (dense), B_{p+1} = Q_p^T B_p Q_p; pass p's map must be the
    sequential greedy matching of B_p's graph by strength |b_ij| / sqrt(b_ii b_jj)
    (integer weights: every product exact, the strength rounded once per IEEE
    operation on both sides), numbered by representatives."""
    from helpers import dense_laplacian, prolongation
    g = make()
    h = orc.Hierarchy(g, passes=passes, coarse_max=8)
    assert h.status == 0 and h.n_levels >= 3
    Ak = dense_laplacian(g)
    for k in range(h.n_levels - 1):
        B = Ak
        maps = h.level_pass_aggs(k)
        assert len(maps) == passes
        for a in maps:
            n = B.shape[0]
            rows, cols = np.nonzero(B - np.diag(np.diag(B)))
            rowptr = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=n))]).astype(np.int64)
            s = -B[rows, cols] / np.sqrt(np.diag(B)[rows] * np.diag(B)[cols])
            inter = gg.Graph(n, rowptr, cols.astype(np.int32), s, None)
            mate = greedy_matching(inter, 0)
            assert np.array_equal(a, numbered_by_representatives(mate))
            Q = prolongation(a, a.max() + 1)
            B = Q.T @ B @ Q
        assert np.array_equal(B, h.level_dense(k + 1))
        Ak = B
