"""Pins of the oracle's stationary AMLI cycle and of the automatic smoother
degree (Sec. 4; Eq. bound-on-m, Sec. 3).

* The AMLI W-cycle applied to unit vectors equals the dense recursion built
  bottom-up from the hierarchy's matrices: B_{L-1} = A_c^+, and for k < L-1
  B_k = Rbar + (I - R A) P Q P^T (I - A R), Rbar = 2R - RAR, with
  Q = A_{k+1}^+ on the coarsest level and Q = q(B_{k+1} A_{k+1}) B_{k+1}
  above it (q read back from the hierarchy, then checked against Remez).  The dense side evaluates q in the monomial basis (numpy's
  Chebyshev-to-power conversion on [alpha, 1]) with matrix powers, the
  smoother by an eigen-decomposition: no step shares the oracle's vector
  recurrences, so a wrong coefficient, index, sign, level or a dropped
  smoothing step fails it.
* B_0 is symmetric and positive definite on 1-perp and the spectrum of B_0 A
  lies in (0, 1] (the point of the positivity condition and of scaling q by
  1/(1 + E)).
* The automatic degree is the smallest m whose best-approximation error,
  measured by Remez exchange, is at most rho (and below 1).
"""
import numpy as np
import pytest
from numpy.polynomial import Chebyshev

import graphgen as gg
from helpers import cheb_q, matrix_function, prolongation, random_graph


def dense_amli(orc, h, alpha, nu):
    L = h.n_levels
    A = [h.level_dense(k) for k in range(L)]
    pw = Chebyshev(h.amli_coef(), domain=[alpha, 1.0]).convert(kind=np.polynomial.Polynomial).coef
    assert pw.size == nu  # degree nu - 1
    M = np.linalg.pinv(A[L - 1], rcond=1e-12, hermitian=True)  # B_{L-1}
    for k in range(L - 2, -1, -1):
        Ak = A[k]
        l0, l1 = h.level_lambda(k)
        R = matrix_function(Ak, lambda lam: cheb_q(h.level_cheb(k), l0, l1, lam))
        agg = h.level_agg(k)
        P = prolongation(agg, agg.max() + 1)
        if k + 1 == L - 1:
            Q = M
        else:
            X = M @ A[k + 1]
            q = np.zeros_like(X)
            Xp = np.eye(X.shape[0])
            for c in pw:                 # sum_i p_i X^i
                q += c * Xp
                Xp = Xp @ X
            Q = q @ M
        I = np.eye(Ak.shape[0])
        M = 2 * R - R @ Ak @ R + (I - R @ Ak) @ P @ Q @ P.T @ (I - Ak @ R)
    return M


GRAPHS = {
    "grid2d_16": lambda: gg.grid2d_5pt(16),
    "grid3d_7_d": lambda: gg.grid3d_7pt(7, 1.0),
    "rand_w": lambda: random_graph(180, 0.03, 7, wmax=4, d_frac=0.05),
}


@pytest.mark.parametrize("nu,alpha", [(2, 0.25), (2, 0.4), (3, 0.15)])
@pytest.mark.parametrize("gname", sorted(GRAPHS))
def test_amli_cycle_is_dense_recursion(orc, gname, nu, alpha):
    g = GRAPHS[gname]()
    h = orc.Hierarchy(g, degree=3, passes=1, coarse_max=12, cycle=1, amli_alpha=alpha, inner_iters=nu)
    assert h.status == 0
    assert h.n_levels >= 4          # at least two levels use the polynomial
    B = dense_amli(orc, h, alpha, nu)
    Bcyc = np.column_stack([h.amli_cycle(0, e) for e in np.eye(g.n)])
    assert np.abs(Bcyc - B).max() <= 1e-10 * np.abs(B).max()


@pytest.mark.parametrize("gname", sorted(GRAPHS))
def test_amli_preconditioner_is_spd(orc, gname):
    g = GRAPHS[gname]()
    h = orc.Hierarchy(g, degree=4, passes=1, coarse_max=12, cycle=1)
    B = np.column_stack([h.amli_cycle(0, e) for e in np.eye(g.n)])
    assert np.abs(B - B.T).max() <= 1e-11 * np.abs(B).max()
    A = h.level_dense(0)
    n = g.n
    Z = np.eye(n)
    if gg.is_pure_laplacian(g):   # restrict to 1-perp
        Z = np.linalg.qr(np.column_stack([np.ones(n), np.eye(n)[:, : n - 1]]))[0][:, 1:]
    Bz, Az = Z.T @ B @ Z, Z.T @ A @ Z
    assert np.linalg.eigvalsh((Bz + Bz.T) / 2).min() > 0
    # spectrum of BA (similar to Lh' B Lh, Az = Lh Lh') in (0, 1]
    Lh = np.linalg.cholesky(Az)
    ev = np.linalg.eigvalsh(Lh.T @ ((Bz + Bz.T) / 2) @ Lh)
    assert ev.min() > 0 and ev.max() <= 1 + 1e-10


def test_amli_rejects_indefinite_polynomial(orc):
    g = gg.grid3d_7pt(6, 1.0)
    # degree-1 approximation on [0.1, 1]: error delta (kappa - 1)/2 = 2.34 >= 1
    assert orc.Hierarchy(g, cycle=1, amli_alpha=0.1, inner_iters=2).status != 0
    # degree 0 on [0.25, 1]: error (kappa - 1)/2 = 1.5
    assert orc.Hierarchy(g, cycle=1, amli_alpha=0.25, inner_iters=1).status != 0
    assert orc.Hierarchy(g, cycle=1, amli_alpha=0.25, inner_iters=2).status == 0


@pytest.mark.parametrize("g,opts", [
    (gg.grid2d_5pt(64), dict(degree=3, passes=2)),
    (gg.grid3d_7pt(20, 1.0), dict(degree=5, passes=3)),
    (gg.grid2d_random_diag(40, 3), dict(degree=4, passes=3)),
])
def test_amli_pcg_converges(orc, g, opts):
    b = gg.rhs(g.n, 21, gg.is_pure_laplacian(g))
    r = orc.Hierarchy(g, cycle=1, **opts).solve(b, tol=1e-8)
    k = orc.Hierarchy(g, **opts).solve(b, tol=1e-8)
    assert r.status == 0 and r.iterations <= k.iterations + 4
    from helpers import sparse_laplacian
    A = sparse_laplacian(g)
    assert np.linalg.norm(b - A @ r.x) <= 1e-7 * np.linalg.norm(b)


@pytest.mark.parametrize("ratio", [0.05, 0.1, 0.2])
@pytest.mark.parametrize("rho", [0.6, 1 / 3, 0.1, 0.01])
def test_degree_from_bound_on_m_matches_remez(orc, ratio, rho):
    m = orc.degree_for(rho, ratio)
    assert m >= 0

    def E(mm):  # lambda1 * max |1/x - q_mm| on [ratio, 1], lambda1 = 1
        return orc.remez_inverse(mm, ratio, 1.0)[1]

    assert E(m) <= rho * (1 + 1e-9) and E(m) < 1
    if m > 0:
        assert E(m - 1) > rho * (1 - 1e-9) or E(m - 1) >= 1


def test_degree_consistent_with_section4(orc):
    # Sec. 4: with lambda0 = lambda1/10, m = 4 satisfies the bound; under the
    # reading E_m <= rho this holds for rho = 1/3 and m = 3 does not suffice
    assert orc.degree_for(1 / 3, 0.1) == 4
    assert orc.degree_for(0.0, 0.1) == -1


def test_rho_sets_the_hierarchy_degree(orc):
    g = gg.grid3d_7pt(10, 1.0)
    h = orc.Hierarchy(g, rho=0.1, degree=2)
    assert h.status == 0 and h.opts.degree == orc.degree_for(0.1, 0.1)
    l0, l1 = h.level_lambda(0)
    ref = orc.remez_inverse(h.opts.degree, l0, l1)[0]
    assert np.allclose(h.level_cheb(0), ref, rtol=0, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("nu,alpha", [(2, 0.25), (3, 0.15)])
def test_amli_polynomial_is_scaled_best_approximation(orc, nu, alpha):
    g = gg.grid3d_7pt(8, 1.0)
    h = orc.Hierarchy(g, cycle=1, amli_alpha=alpha, inner_iters=nu)
    c, err, _ = orc.remez_inverse(nu - 1, alpha, 1.0)
    kappa = 1 / alpha
    delta = (np.sqrt(kappa) - 1) / (np.sqrt(kappa) + 1)
    E = delta ** (nu - 1) * (kappa - 1) / 2
    assert err == pytest.approx(E, rel=1e-10)           # Sec. 3 with lambda1 = 1
    assert np.allclose(h.amli_coef(), c / (1 + E), rtol=1e-12, atol=0)
    t = np.linspace(alpha, 1, 2001)
    tq = t * Chebyshev(h.amli_coef(), domain=[alpha, 1.0])(t)
    assert tq.max() <= 1 + 1e-12 and tq.min() > 0


@pytest.mark.parametrize("nu,alpha", [(2, 0.25), (3, 0.15)])
def test_amli_cycle_is_dense_recursion_on_independent_set_aggregates(orc, nu, alpha):
    """The same dense recursion on a hierarchy built by the paper's aggregation
    (maximal independent sets of the graph of A^k, Sec. 2; k = 1 keeps five
    levels on a 20 x 20 grid): the cycle depends on the aggregates only through
    P and the Galerkin operators."""
    g = gg.grid2d_5pt(20)
    h = orc.Hierarchy(g, degree=3, passes=1, coarse_max=12, cycle=1, amli_alpha=alpha, inner_iters=nu,
                      aggregation=1, mis_k=1)
    assert h.status == 0 and h.n_levels >= 4
    B = dense_amli(orc, h, alpha, nu)
    Bcyc = np.column_stack([h.amli_cycle(0, e) for e in np.eye(g.n)])
    assert np.abs(Bcyc - B).max() <= 1e-10 * np.abs(B).max()


@pytest.mark.parametrize("R", [1, 5])
@pytest.mark.parametrize("gname", ["grid3d_7_d", "rand_w"])
def test_amli_solve_is_restarted_pcg_with_dense_B(orc, gname, R):
    """The stationary AMLI cycle is a fixed linear SPD operator B_0, so the
    outer flexible CG preconditioned by it (Sec. 4, restarted every R steps)
    has the residual history of textbook PCG with the dense B_0 built by the
    bottom-up recursion."""
    from helpers import restarted_pcg

    g = GRAPHS[gname]()
    iters = 10
    h = orc.Hierarchy(g, degree=3, passes=1, coarse_max=12, cycle=1, restart=R, max_iters=iters)
    assert h.status == 0 and h.n_levels >= 4
    B = dense_amli(orc, h, 0.25, 2)
    b = gg.rhs(g.n, 33, False)
    res = h.solve(b, tol=1e-30)
    ref = restarted_pcg(h.level_dense(0), B, b, R, iters)
    assert len(res.history) == iters + 1
    assert np.allclose(res.history, ref, rtol=1e-7, atol=1e-13)
