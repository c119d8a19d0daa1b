"""Pins of the oracle's single-step operations, the ones the device parity
tests compare against one by one.

* SpMV at level k: the product with the operator assembled from the graph
  (Eq. (1)) at level 0 and with the dense Galerkin product P^T A P built from
  the aggregate maps (Sec. 2 Eq. (coarse)) on the levels below; no step reads
  the oracle's stored matrices.
* Restriction r_H = P^T s and prolongation x + P e_H (Sec. 2) on integer
  vectors, where every sum is exact: equality bit for bit with the dense
  0/1 prolongation matrix.
* The inner solve of nu flexible-CG steps at level k = L-2, whose
  preconditioner is the linear two-level operator B (exact coarse solve,
  Sec. 3): nu PCG steps, i.e. the A-orthogonal projection onto the Krylov
  space K_nu(BA, Bb), for nu = 1, 2, 3.
* The smoother interval of every smoothed level: lambda1 = ||A_k||_inf from
  the dense chain, an upper bound on lambda_max, and lambda0 = lambda1 / 10
  (or the configured ratio, with the Remez coefficients of that interval).
* Pure Laplacians: the constant part of b does not change the solution, which
  has zero mean.
"""
import numpy as np
import pytest

import graphgen as gg
from helpers import cheb_q, dense_laplacian, matrix_function, prolongation, random_graph

GRAPHS = {
    "grid2d_14": lambda: gg.grid2d_5pt(14),
    "grid3d_6_d": lambda: gg.grid3d_7pt(6, 1.0),
    "rand_w": lambda: random_graph(220, 0.025, 3, wmax=4, d_frac=0.05),
}


def hierarchy(orc, g, **kw):
    h = orc.Hierarchy(g, degree=3, passes=1, coarse_max=12, **kw)
    assert h.status == 0 and h.n_levels >= 3
    return h


def galerkin_chain(h, g):
    """Dense operators of every level from the graph and the aggregate maps."""
    A = [dense_laplacian(g)]
    for k in range(h.n_levels - 1):
        P = prolongation(h.level_agg(k), h.level_n(k + 1))
        A.append(P.T @ A[-1] @ P)
    return A


@pytest.mark.parametrize("gname", sorted(GRAPHS))
def test_spmv_is_assembled_operator(orc, gname):
    g = GRAPHS[gname]()
    h = hierarchy(orc, g)
    rng = np.random.default_rng(7)
    for k, Ak in enumerate(galerkin_chain(h, g)):
        x = rng.standard_normal(Ak.shape[0])
        y = Ak @ x
        assert np.abs(h.spmv(k, x) - y).max() <= 1e-13 * np.abs(Ak).max() * np.abs(x).sum()
        xi = rng.integers(-50, 50, Ak.shape[0]).astype(float)   # integer data: exact sums
        assert np.array_equal(h.spmv(k, xi), Ak @ xi)


@pytest.mark.parametrize("gname", sorted(GRAPHS))
def test_transfers_are_the_piecewise_constant_prolongation(orc, gname):
    g = GRAPHS[gname]()
    h = hierarchy(orc, g)
    rng = np.random.default_rng(8)
    for k in range(h.n_levels - 1):
        n, nH = h.level_n(k), h.level_n(k + 1)
        P = prolongation(h.level_agg(k), nH)
        assert np.array_equal(P.sum(axis=1), np.ones(n))        # each vertex in one aggregate
        s = rng.integers(-1000, 1000, n).astype(float)
        assert np.array_equal(h.restrict(k, s), P.T @ s)
        e = rng.integers(-1000, 1000, nH).astype(float)
        x = rng.integers(-1000, 1000, n).astype(float)
        assert np.array_equal(h.prolong_add(k, e, x), x + P @ e)
        # adjointness: (P^T s, e) = (s, P e)
        assert h.restrict(k, s) @ e == s @ (h.prolong_add(k, e, np.zeros(n)))


@pytest.mark.parametrize("nu", [1, 2, 3])
@pytest.mark.parametrize("gname", ["grid2d_14", "rand_w"])
def test_inner_fcg_is_krylov_projection(orc, gname, nu):
    g = GRAPHS[gname]()
    h = orc.Hierarchy(g, degree=3, passes=1, coarse_max=g.n // 7, max_levels=3, inner_iters=nu)
    assert h.status == 0 and h.n_levels == 3
    A = galerkin_chain(h, g)
    A1, A2 = A[1], A[2]
    l0, l1 = h.level_lambda(1)
    R = matrix_function(A1, lambda lam: cheb_q(h.level_cheb(1), l0, l1, lam))
    P = prolongation(h.level_agg(1), A2.shape[0])
    I = np.eye(A1.shape[0])
    B = 2 * R - R @ A1 @ R + (I - R @ A1) @ P @ np.linalg.pinv(A2, rcond=1e-12, hermitian=True) @ P.T @ (I - A1 @ R)
    rng = np.random.default_rng(9)
    for _ in range(3):
        b = rng.standard_normal(A1.shape[0])
        if gg.is_pure_laplacian(g):
            b -= b.mean()
        cols = [B @ b]
        for _ in range(nu - 1):
            cols.append(B @ (A1 @ cols[-1]))
        V = np.column_stack(cols)
        x = V @ np.linalg.solve(V.T @ A1 @ V, V.T @ b)
        got = h.inner_fcg(1, b)
        # compare in the A_1 energy norm (the quantity CG minimises; insensitive
        # to the constant vector's component on pure Laplacians)
        d = got - x
        assert np.sqrt(d @ A1 @ d) <= 1e-9 * np.sqrt(x @ A1 @ x)


@pytest.mark.parametrize("gname", sorted(GRAPHS))
def test_smoother_interval_on_every_level(orc, gname):
    """lambda1 = ||A_k||_inf (a Gershgorin bound on lambda_max, Sec. 3) and
    lambda0 = lambda1 / 10 (Sec. 4) on every smoothed level, from the dense
    Galerkin chain; integer weights make the row sums exact."""
    g = GRAPHS[gname]()
    h = hierarchy(orc, g)
    A = galerkin_chain(h, g)
    for k in range(h.n_levels - 1):
        l0, l1 = h.level_lambda(k)
        assert l1 == np.abs(A[k]).sum(axis=1).max()
        assert np.linalg.eigvalsh(A[k])[-1] <= l1 * (1 + 1e-14)
        assert l0 == pytest.approx(0.1 * l1, rel=1e-15)


@pytest.mark.parametrize("ratio", [0.05, 0.2])
def test_smoother_interval_follows_lambda0_ratio(orc, ratio):
    """lambda0 = ratio * lambda1 for a non-default ratio, and the stored
    coefficients are the best approximation on that interval (Remez, Sec. 3)."""
    g = GRAPHS["rand_w"]()
    h = orc.Hierarchy(g, degree=4, passes=1, coarse_max=12, lambda0_ratio=ratio)
    assert h.status == 0
    for k in range(h.n_levels - 1):
        l0, l1 = h.level_lambda(k)
        assert l0 == pytest.approx(ratio * l1, rel=1e-15)
        ref = orc.remez_inverse(4, l0, l1)[0]
        assert np.allclose(h.level_cheb(k), ref, rtol=0, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("gname", ["grid2d_14", "rand_w"])
def test_pure_laplacian_ignores_the_constant_part_of_b(orc, gname):
    """The range of a pure Laplacian is 1-perp (Sec. 1): b and b + c 1 give the
    same solution, which has zero mean; with a lower-order term they differ."""
    g = GRAPHS[gname]()
    h = orc.Hierarchy(g, degree=3, passes=2, coarse_max=12)
    b = gg.rhs(g.n, 41, True)
    x1 = h.solve(b, tol=1e-12).x
    x2 = h.solve(b + 5.0, tol=1e-12).x
    if gg.is_pure_laplacian(g):
        assert np.allclose(x1, x2, rtol=0, atol=1e-10 * np.abs(x1).max())
        assert abs(x1.mean()) <= 1e-12 * np.abs(x1).max()
    else:
        A = dense_laplacian(g)
        assert np.linalg.norm(A @ x2 - (b + 5.0)) <= 1e-10 * np.linalg.norm(b + 5.0)
        assert not np.allclose(x1, x2)
