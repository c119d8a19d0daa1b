"""Pins of the oracle's smoother: the polynomial of best uniform approximation to
1/x (Eq. (1x-1-min)) computed by Remez exchange, and its application q_m(A) r by
the Chebyshev recurrence."""
import os

import numpy as np
import pytest

import graphgen as gg
from helpers import cheb_q, dense_laplacian, matrix_function, random_graph

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def closed_form_E(m, kappa):
    """Paper, Sec. 3: E_m = delta^m (kappa - 1) / 2."""
    delta = (np.sqrt(kappa) - 1) / (np.sqrt(kappa) + 1)
    return delta ** m * (kappa - 1) / 2


def closed_form_coefficients(m, l0, l1):
    """Chebyshev coefficients of the best approximation, derived independently of
    Remez: with 1/x = 2/(l1-l0) * 1/(t+a), a = (l1+l0)/(l1-l0), delta = a - sqrt(a^2-1),
    the error of the best degree-m approximant of 1/(t+a) is E*Re(z^m B(z)),
    B(z) = (z+delta)/(1+delta z), z = e^{i theta}; matching the poles of 1/(t+a)
    gives c_k = 4 delta (-delta)^k / (1-delta^2) (k < m, c_0 halved) and
    c_m = (-1)^m 4 delta^(m+1) / (1-delta^2)^2 (m >= 1);
    m = 0: c_0 = 2 delta (1+delta^2)/(1-delta^2)^2, the midpoint of 1/(a+-1)."""
    a = (l1 + l0) / (l1 - l0)
    dl = a - np.sqrt(a * a - 1)
    c = np.zeros(m + 1)
    if m == 0:
        c[0] = 2 * dl * (1 + dl * dl) / (1 - dl * dl) ** 2
    else:
        c[0] = 2 * dl / (1 - dl * dl)
        for k in range(1, m):
            c[k] = 4 * dl * (-dl) ** k / (1 - dl * dl)
        c[m] = (-1) ** m * 4 * dl ** (m + 1) / (1 - dl * dl) ** 2
    return c * 2.0 / (l1 - l0)


def test_degree_zero_closed_form(orc):
    l0, l1 = 0.7, 7.0
    c, err, alt = orc.remez_inverse(0, l0, l1)
    assert c[0] == pytest.approx((1 / l0 + 1 / l1) / 2, rel=1e-15)
    assert err == pytest.approx((1 / l0 - 1 / l1) / 2, rel=1e-15)


@pytest.mark.parametrize("kappa", [2.0, 10.0, 30.0, 100.0])
@pytest.mark.parametrize("m", list(range(0, 11)))
def test_error_matches_paper_closed_form(orc, m, kappa):
    l1 = 12.0
    l0 = l1 / kappa
    c, err, alt = orc.remez_inverse(m, l0, l1)
    # E_m = lambda1 * max|1/x - q_m| since lambda1 is an alternance point (Sec. 3)
    assert l1 * err == pytest.approx(closed_form_E(m, kappa), rel=1e-12)


def test_golden_values_kappa10(orc):
    rows = [l.split() for l in open(os.path.join(GOLD, "smoother_error_kappa10.txt")) if l[0] != "#"]
    for m, Em in rows:
        c, err, _ = orc.remez_inverse(int(m), 1.0, 10.0)
        assert round(10.0 * err, 5) == pytest.approx(float(Em), abs=5e-6)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 7, 10])
def test_equioscillation(orc, m):
    """Chebyshev alternation: m+2 points incl. l0 and l1 where the error is
    +-E with alternating signs, and |error| <= E everywhere on [l0, l1]."""
    l0, l1 = 0.5, 5.0
    c, err, alt = orc.remez_inverse(m, l0, l1)
    assert alt[0] == pytest.approx(l0, rel=1e-12) and alt[-1] == pytest.approx(l1, rel=1e-12)
    e = 1 / alt - cheb_q(c, l0, l1, alt)
    assert np.allclose(np.abs(e), err, rtol=1e-9)
    assert np.all(np.sign(e[:-1]) == -np.sign(e[1:]))
    xs = np.linspace(l0, l1, 20001)
    assert np.max(np.abs(1 / xs - cheb_q(c, l0, l1, xs))) <= err * (1 + 1e-9)


@pytest.mark.parametrize("m", [0, 1, 2, 3, 4, 5, 6, 9])
@pytest.mark.parametrize("kappa", [10.0, 40.0])
def test_coefficients_match_independent_derivation(orc, m, kappa):
    l1 = 9.0
    l0 = l1 / kappa
    c, err, _ = orc.remez_inverse(m, l0, l1)
    cf = closed_form_coefficients(m, l0, l1)
    assert np.allclose(c, cf, rtol=1e-11, atol=1e-13 * np.abs(cf).max())


@pytest.mark.parametrize("m", [3, 4, 5, 6])
def test_positivity_and_damping_on_0_l1(orc, m):
    """Sec. 3: q_m(l1) > 0 once E_m < 1, making R = q_m(A) SPD; the spectrum of A
    reaches below l0, so also check q_m > 0 and |1 - x q_m(x)| <= 1 on [0, l1]."""
    l1 = 8.0
    l0 = l1 / 10
    c, err, _ = orc.remez_inverse(m, l0, l1)
    xs = np.linspace(0.0, l1, 40001)
    q = cheb_q(c, l0, l1, xs)
    assert np.all(q > 0)
    assert np.all(np.abs(1 - xs * q) <= 1 + 1e-12)


@pytest.mark.parametrize("m", [0, 1, 3, 5])
def test_smoother_application_matches_dense_matrix_function(orc, m):
    g = random_graph(60, 0.08, seed=11, wmax=3, d_frac=0.1)
    h = orc.Hierarchy(g, degree=m, passes=1, coarse_max=8)
    assert h.status == 0 and h.n_levels >= 2
    A = dense_laplacian(g)
    l0, l1 = h.level_lambda(0)
    assert l1 == pytest.approx(np.abs(A).sum(axis=1).max(), rel=1e-15)  # ||A||_inf, Sec. 3
    assert l0 == pytest.approx(l1 / 10, rel=1e-15)                     # Sec. 4
    coef = h.level_cheb(0)
    c_ref, _, _ = orc.remez_inverse(m, l0, l1)
    assert np.array_equal(coef, c_ref)
    R = matrix_function(A, lambda lam: cheb_q(coef, l0, l1, lam))
    r = gg.uniform_pm1(5, g.n)
    assert np.allclose(h.smooth(0, r), R @ r, rtol=1e-11, atol=1e-11 * np.abs(R @ r).max())
