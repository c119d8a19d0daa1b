"""Pins of the oracle's cycle and Krylov solver.

* Two levels: the symmetric W(1,1) cycle (pre-smooth, exact coarse correction
  with A_H^+, post-smooth) is the paper's symmetrised two-level preconditioner
  B, whose closed form is B = Rbar + (I - RA) P A_H^+ P^T (I - AR),
  Rbar = 2R - RAR (Sec. 3).  Also lambda_max(BA) <= 1 on 1-perp (lower half
  of the spectral equivalence) and ||E_TL||_A^2 = rho(I - BA).
* Exact solves with known answers: path graph, complete graph, dense pinv.
* Special cases: identity preconditioner + no restart = textbook CG; exact
  preconditioner converges in one iteration.
"""
import numpy as np
import pytest

import graphgen as gg
from helpers import (cheb_q, complete_graph, dense_laplacian, matrix_function, path_graph,
                     prolongation, random_graph, restarted_pcg)


def two_level(orc, g, m):
    h = orc.Hierarchy(g, degree=m, passes=2, coarse_max=g.n // 3, max_levels=2)
    assert h.status == 0 and h.n_levels == 2
    return h


def dense_B(orc, h, g, m):
    A = dense_laplacian(g)
    l0, l1 = h.level_lambda(0)
    R = matrix_function(A, lambda lam: cheb_q(h.level_cheb(0), l0, l1, lam))
    agg = h.level_agg(0)
    P = prolongation(agg, agg.max() + 1)
    AH = P.T @ A @ P
    I = np.eye(g.n)
    Rbar = 2 * R - R @ A @ R
    B = Rbar + (I - R @ A) @ P @ np.linalg.pinv(AH, rcond=1e-12, hermitian=True) @ P.T @ (I - A @ R)
    return A, R, P, AH, B


@pytest.mark.parametrize("m", [1, 2, 3, 4, 6])
@pytest.mark.parametrize("gname", ["grid", "rand"])
def test_two_level_cycle_is_closed_form_B(orc, m, gname):
    g = gg.grid2d_5pt(9) if gname == "grid" else random_graph(70, 0.06, 2, wmax=3)
    h = two_level(orc, g, m)
    A, R, P, AH, B = dense_B(orc, h, g, m)
    Bcyc = np.column_stack([h.kcycle(0, e) for e in np.eye(g.n)])
    assert np.allclose(Bcyc, B, rtol=1e-10, atol=1e-10 * np.abs(B).max())


@pytest.mark.parametrize("gname", ["grid", "rand"])
def test_two_level_spectral_bounds(orc, gname):
    g = gg.grid2d_5pt(9) if gname == "grid" else random_graph(70, 0.06, 2, wmax=3)
    kappas = []
    # Eq. (bound-on-m): the bound needs E_m < 1, i.e. m >= 3 for kappa = 10
    for m in [3, 4, 5, 6]:
        h = two_level(orc, g, m)
        A, R, P, AH, B = dense_B(orc, h, g, m)
        n = g.n
        # restrict to 1-perp with an orthonormal basis Z of the complement of 1
        Z = np.linalg.qr(np.column_stack([np.ones(n), np.eye(n)[:, : n - 1]]))[0][:, 1:]
        Ar = Z.T @ A @ Z
        Lh = np.linalg.cholesky(Ar)
        M = Lh.T @ (Z.T @ B @ Z) @ Lh                          # similar to BA on 1-perp
        ev = np.linalg.eigvalsh((M + M.T) / 2)
        assert ev.max() <= 1 + 1e-10                           # v'Av <= v'B^+v
        assert ev.min() > 0
        # ||E_TL||_A^2 = rho(I - BA), E_TL = (I - RA)(I - pi_A), pi_A = P A_H^+ P^T A
        pi = P @ np.linalg.pinv(AH, rcond=1e-12, hermitian=True) @ P.T @ A
        E = (np.eye(n) - R @ A) @ (np.eye(n) - pi)
        Er = Lh.T @ (Z.T @ E @ Z) @ np.linalg.inv(Lh.T)      # A^{1/2} E A^{-1/2} in 1-perp
        assert np.linalg.norm(Er, 2) ** 2 == pytest.approx(max(abs(1 - ev)), rel=1e-8)
        kappas.append(ev.max() / ev.min())
    assert all(k2 <= k1 * (1 + 1e-9) for k1, k2 in zip(kappas, kappas[1:]))


def test_path_graph_linear_solution(orc):
    n = 50
    g = path_graph(n)
    h = orc.Hierarchy(g, degree=3, passes=2, coarse_max=4)
    b = np.zeros(n); b[0], b[-1] = 1.0, -1.0
    r = h.solve(b, tol=1e-12)
    assert r.status == 0
    assert np.allclose(np.diff(r.x), -1.0, atol=1e-9)
    assert abs(r.x.mean()) < 1e-12


def test_complete_graph(orc):
    n = 120
    g = complete_graph(n)
    h = orc.Hierarchy(g, degree=3, passes=2, coarse_max=8)
    b = gg.rhs(n, 7, True)
    r = h.solve(b, tol=1e-12)
    assert r.status == 0
    assert np.allclose(r.x, b / n, rtol=0, atol=1e-11 * np.abs(b / n).max())


@pytest.mark.parametrize("seed", range(4))
def test_solution_equals_dense_pinv(orc, seed):
    g = random_graph(200, 0.02, seed, wmax=4, d_frac=0.05 if seed % 2 else 0.0)
    h = orc.Hierarchy(g, degree=4, passes=2, coarse_max=12)
    assert h.status == 0 and h.n_levels >= 3
    A = dense_laplacian(g)
    b = gg.rhs(g.n, 100 + seed, g.d is None)
    r = h.solve(b, tol=1e-10)
    assert r.status == 0 and r.history[-1] <= 1e-10
    xs = np.linalg.pinv(A, rcond=1e-12, hermitian=True) @ b
    ev = np.linalg.eigvalsh(A)
    kappa = ev[-1] / ev[ev > 1e-9 * ev[-1]][0]
    assert np.linalg.norm(r.x - xs) <= 1e-9 * kappa * np.linalg.norm(xs)
    assert r.true_rel_residual == pytest.approx(np.linalg.norm(b - A @ r.x) / np.linalg.norm(b), rel=1e-6)


def test_identity_preconditioner_is_textbook_cg(orc):
    g = gg.grid2d_5pt(12)
    b = gg.rhs(g.n, 3, True)
    h = orc.Hierarchy(g, precond=orc.PREC_IDENTITY, restart=10 ** 6, max_iters=25)
    r = h.solve(b, tol=1e-30)
    A = dense_laplacian(g)
    x = np.zeros(g.n); rr = b.copy(); p = rr.copy(); hist = [1.0]
    for _ in range(25):                                        # Hestenes-Stiefel CG
        Ap = A @ p
        a = (rr @ rr) / (p @ Ap)
        x += a * p
        rn = rr - a * Ap
        p = rn + (rn @ rn) / (rr @ rr) * p
        rr = rn
        hist.append(np.linalg.norm(rr) / np.linalg.norm(b))
    assert np.allclose(r.history, hist, rtol=1e-8)


def test_exact_preconditioner_one_iteration(orc):
    g = random_graph(80, 0.05, 5, wmax=2)
    h = orc.Hierarchy(g, precond=orc.PREC_EXACT)
    r = h.solve(gg.rhs(g.n, 9, True), tol=1e-10)
    assert r.status == 0 and r.iterations == 1


def test_coarse_pinv_and_jacobi(orc):
    g = random_graph(40, 0.1, 8, wmax=3)
    A = dense_laplacian(g)
    ev, V = orc.jacobi_eigen(A)
    assert np.allclose(np.sort(ev), np.linalg.eigvalsh(A), atol=1e-12 * ev.max())
    assert np.allclose(V @ np.diag(ev) @ V.T, A, atol=1e-12 * ev.max())
    h = orc.Hierarchy(g, coarse_max=10 ** 6)
    b = gg.uniform_pm1(4, g.n)                                 # not zero-mean: pinv projects
    assert np.allclose(h.coarse_solve(b), np.linalg.pinv(A, rcond=1e-12, hermitian=True) @ b, atol=1e-12)


def test_history_and_stopping(orc):
    g = gg.grid3d_7pt(10, 1.0)
    h = orc.Hierarchy(g, degree=5, passes=3)
    r = h.solve(gg.rhs(g.n, 2, False), tol=1e-8)
    assert r.status == 0 and r.converged
    assert r.history[0] == 1.0 and r.history[-1] <= 1e-8 < r.history[-2]
    assert len(r.history) == r.iterations + 1
    assert r.true_rel_residual < 1e-7
    r2 = orc.Hierarchy(g, degree=5, passes=3, max_iters=2).solve(gg.rhs(g.n, 2, False))
    assert r2.status == orc.ERR_NOT_CONVERGED and r2.iterations == 2


@pytest.mark.parametrize("gname", ["grid", "rand", "grid_mis"])
def test_kcycle_inner_fcg_is_krylov_projection(orc, gname):
    """Three levels: the preconditioner of the inner solve at level 1 is the
    linear two-level operator M = B_1 (exact coarse solve at level 2), so nu = 2
    flexible-CG steps are two PCG steps and their result is the A_1-orthogonal
    projection of A_1^{-1} r_H onto K_2 = span{M r_H, M A_1 M r_H}: e_H =
    V (V' A_1 V)^{-1} V' r_H (the optimality of CG, Sec. 4's NPCG on a linear
    preconditioner).  The K-cycle at level 0 is then the two-level sweep of
    Sec. 3 with that e_H."""
    g = gg.grid2d_5pt(24) if gname.startswith("grid") else random_graph(500, 0.01, 6, wmax=3, d_frac=0.05)
    agg = dict(aggregation=1, mis_k=1) if gname.endswith("mis") else {}
    h = orc.Hierarchy(g, degree=3, passes=1, coarse_max=g.n // 7, max_levels=3, inner_iters=2, **agg)
    assert h.status == 0 and h.n_levels == 3
    A0, A1, A2 = (h.level_dense(k) for k in range(3))
    def smoother(k, A):
        l0, l1 = h.level_lambda(k)
        return matrix_function(A, lambda lam: cheb_q(h.level_cheb(k), l0, l1, lam))
    R0, R1 = smoother(0, A0), smoother(1, A1)
    P0 = prolongation(h.level_agg(0), A1.shape[0])
    P1 = prolongation(h.level_agg(1), A2.shape[0])
    I1 = np.eye(A1.shape[0])
    M = (2 * R1 - R1 @ A1 @ R1
         + (I1 - R1 @ A1) @ P1 @ np.linalg.pinv(A2, rcond=1e-12, hermitian=True) @ P1.T @ (I1 - A1 @ R1))
    rng = np.random.default_rng(4)
    for _ in range(3):
        r = rng.standard_normal(g.n)
        if gg.is_pure_laplacian(g):
            r -= r.mean()
        u = R0 @ r
        rH = P0.T @ (r - A0 @ u)
        V = np.column_stack([M @ rH, M @ A1 @ (M @ rH)])
        eH = V @ np.linalg.solve(V.T @ A1 @ V, V.T @ rH)
        x = u + P0 @ eH
        x = x + R0 @ (r - A0 @ x)
        got = h.kcycle(0, r)
        assert np.abs(got - x).max() <= 1e-9 * np.abs(x).max()


@pytest.mark.parametrize("R", [1, 3, 5])
@pytest.mark.parametrize("pre", ["identity", "two_level"])
def test_restarted_flexible_cg_is_restarted_pcg(orc, pre, R):
    """With a fixed SPD preconditioner the window's orthogonalisation reduces
    to PCG's one-term recurrence (Sec. 4 restarts the outer iteration every
    five steps); R = 1 with the identity is steepest descent.  Pins the window
    reset index, the projection coefficients and the step length."""
    g = random_graph(90, 0.05, 11, wmax=3, d_frac=0.05)
    b = gg.rhs(g.n, 31, False)
    iters = 12
    if pre == "identity":
        h = orc.Hierarchy(g, precond=orc.PREC_IDENTITY, restart=R, max_iters=iters)
        A, B = dense_laplacian(g), np.eye(g.n)
    else:
        h = orc.Hierarchy(g, degree=3, passes=2, coarse_max=g.n // 3, max_levels=2, restart=R,
                          max_iters=iters)
        assert h.status == 0 and h.n_levels == 2
        A, _, _, _, B = dense_B(orc, h, g, 3)
    res = h.solve(b, tol=1e-30)
    ref = restarted_pcg(A, B, b, R, iters)
    assert len(res.history) == iters + 1
    assert np.allclose(res.history, ref, rtol=1e-7, atol=1e-13)
