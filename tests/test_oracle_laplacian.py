"""Pins of the oracle's operator assembly (Eq. (1)) and input validation."""
import numpy as np
import pytest

import graphgen as gg
from helpers import dense_laplacian, random_graph, star_graph


@pytest.mark.parametrize("make", [lambda: gg.grid2d_5pt(9), lambda: gg.grid3d_7pt(5, None),
                                  lambda: gg.grid2d_random_diag(8, 3), lambda: random_graph(40, 0.1, 1, wmax=5)])
def test_pure_laplacian_rows_sum_to_zero(orc, make):
    g = make()
    h = orc.Hierarchy(g, coarse_max=10 ** 9)
    assert h.status == 0 and h.n_levels == 1
    A = h.level_dense(0)
    assert np.array_equal(A @ np.ones(g.n), np.zeros(g.n))       # integer weights: exact
    assert np.array_equal(A, A.T)
    assert np.array_equal(A, dense_laplacian(g))
    lam, V = np.linalg.eigh(A)
    assert abs(lam[0]) < 1e-10 * lam[-1] and lam[1] > 1e-8       # kernel = span{1} (Sec. 1)
    v0 = V[:, 0] * np.sign(V[0, 0])
    assert np.allclose(v0, 1 / np.sqrt(g.n), atol=1e-8)


def test_lower_order_term_on_diagonal(orc):
    g = gg.grid3d_7pt(4, 1.0)
    h = orc.Hierarchy(g, coarse_max=10 ** 9)
    rp, col, val, diag, dlow = h.level_csr(0)
    deg = np.diff(g.rowptr).astype(float)
    assert np.array_equal(diag, deg + g.d) and np.array_equal(dlow, g.d)
    assert np.array_equal(val, -g.w)
    assert np.linalg.eigvalsh(h.level_dense(0))[0] > 0           # SPD with d > 0


def _bad(g, **kw):
    return gg.Graph(g.n, kw.get("rowptr", g.rowptr), kw.get("col", g.col), kw.get("w", g.w), kw.get("d", g.d))


def test_validation_codes(orc):
    g = gg.grid2d_5pt(4)
    ok = orc.Hierarchy(g)
    assert ok.status == orc.OK
    w = g.w.copy(); w[3] = 2.0
    assert orc.Hierarchy(_bad(g, w=w)).status == orc.ERR_NOT_SYMMETRIC
    w = -g.w
    assert orc.Hierarchy(_bad(g, w=w)).status == orc.ERR_BAD_WEIGHT
    col = g.col.copy(); col[0] = 0                                 # row 0: (0,0) self loop
    assert orc.Hierarchy(_bad(g, col=col)).status == orc.ERR_SELF_LOOP
    col = g.col.copy(); col[0] = 99
    assert orc.Hierarchy(_bad(g, col=col)).status == orc.ERR_INVALID_ARG
    col = g.col.copy(); col[[0, 1]] = col[[1, 0]]                   # unsorted row
    assert orc.Hierarchy(_bad(g, col=col)).status == orc.ERR_INVALID_ARG
    rp = g.rowptr.copy(); rp[2] = rp[1] - 1
    assert orc.Hierarchy(_bad(g, rowptr=rp)).status == orc.ERR_INVALID_ARG
    d = np.zeros(g.n); d[1] = -1
    assert orc.Hierarchy(_bad(g, d=d)).status == orc.ERR_BAD_WEIGHT
    # two disjoint paths: disconnected pure Laplacian
    two = gg.csr_from_edges(6, np.array([0, 1, 3, 4]), np.array([1, 2, 4, 5]))
    assert orc.Hierarchy(two).status == orc.ERR_DISCONNECTED
    # ... fine once each component has a lower-order term
    two.d = np.array([1.0, 0, 0, 0, 0, 2.0])
    assert orc.Hierarchy(two).status == orc.OK


def test_stall_guard(orc):
    """A star cannot be coarsened by matching (only one leaf pairs with the hub);
    a small star becomes its own coarsest level, a large one is reported."""
    small = orc.Hierarchy(star_graph(200), coarse_max=8)
    assert small.status == orc.OK and small.n_levels == 1
    big = orc.Hierarchy(star_graph(5000), coarse_max=8)
    assert big.status == orc.ERR_SETUP_STALL


def test_oracle_struct_layouts_match_its_header(orc, tmp_path):
    """The oracle's ctypes option and report structures match oracle/amg_oracle.h."""
    import os

    from helpers import assert_layouts_match, c_struct_layouts

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    structs = [("orc_options", orc.Options), ("orc_info", orc.Info)]
    layout = c_struct_layouts(os.path.join(root, "oracle"), "amg_oracle.h", structs, tmp_path)
    if layout is None:
        pytest.skip("no C compiler")
    assert_layouts_match(layout, structs)
