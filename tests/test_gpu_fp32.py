"""GPU checks of the mixed-precision form.

* fp32 preconditioner inside fp64 flexible CG: the outer residual is fp64,
  so every solve still reaches ||r||/||b|| <= 1e-8.  Two solutions that each
  meet that tolerance differ by a vector whose residual is at most 2e-8 ||b||
  (their errors themselves may differ by up to kappa * 1e-8), so that is the
  bound checked against the fp64 oracle's solution; iteration counts stay
  within a few of the fp64 method's.
* fp32 K-cycle applications agree with the fp64 oracle to single-precision
  accuracy (1e-4 relative to the result's max norm).
"""
import numpy as np
import pytest

import graphgen as gg
from helpers import sparse_laplacian

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def amg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1307_6305_gb300 as pkg

    pkg.lib()
    return pkg


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def resid_gap(orc, g, opts, x, xref):
    """||A (x - xref)|| with A assembled from Eq. (1) as a scipy sparse matrix."""
    return np.linalg.norm(sparse_laplacian(g) @ (x - xref))


GRAPHS = {
    "grid3d_24_d": (lambda: gg.grid3d_7pt(24, 1.0), dict(degree=5, passes=3)),
    "rdiag_96": (lambda: gg.grid2d_random_diag(96, 3), dict(degree=4, passes=3)),
    "grid2d_64": (lambda: gg.grid2d_5pt(64), dict(degree=3, passes=2)),
    "rgg_8000": (lambda: gg.random_geometric(8000, 5), dict(degree=4, passes=3)),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_fp32_preconditioner_solve(amg, orc, name):
    make, opts = GRAPHS[name]
    g = make()
    b = gg.rhs(g.n, 13, gg.is_pure_laplacian(g))
    ref = orc.Hierarchy(g, **opts).solve(b, tol=1e-8)
    h = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, precision=amg.AMG_PREC_FP32, **opts)
    assert h.status == 0, h.error
    bd = cuda(b)
    xd = torch.zeros_like(bd)
    st, info, hist = h.solve(bd, xd, tol=1e-8)
    assert st == amg.AMG_OK
    assert hist[-1] <= 1e-8 and info.true_rel_residual < 1e-7
    assert info.iterations <= ref.iterations + 3
    x = xd.cpu().numpy()
    assert resid_gap(orc, g, opts, x, ref.x) <= 2.1e-8 * np.linalg.norm(b)


@pytest.mark.parametrize("name", ["grid3d_24_d", "rdiag_96"])
def test_fp32_kcycle_single_precision_accuracy(amg, orc, name):
    make, opts = GRAPHS[name]
    g = make()
    gh = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, precision=amg.AMG_PREC_FP32, **opts)
    oh = orc.Hierarchy(g, **opts)
    assert gh.status == 0 and gh.n_levels == oh.n_levels
    for k in range(oh.n_levels):
        v = gg.uniform_pm1(300 + k, oh.level_n(k))
        out = torch.zeros(v.size, dtype=torch.float64, device="cuda")
        gh.apply("kcycle", k, cuda(v), out)
        assert rel(out.cpu().numpy(), oh.kcycle(k, v)) < 1e-4
        if k + 1 < oh.n_levels:
            out.zero_()
            gh.apply("smoother", k, cuda(v), out)
            assert rel(out.cpu().numpy(), oh.smooth(k, v)) < 1e-5


@pytest.mark.slow
def test_full_size_rdiag_2048_fp32(amg, orc):
    """The mixed-precision workload at full size: 2048^2 random-diagonal
    triangulation, pure Laplacian, degree 4, three passes per level, fp32
    preconditioner in fp64 flexible CG.  Reports the final error against the
    fp64 oracle and the iterations against the plain fp64 GPU run."""
    g, p = gg.workload("rdiag2d_2048")
    b = gg.rhs(g.n, p["rhs_seeds"][0], True)
    opts = dict(degree=p["degree"], passes=p["passes"])
    ref = orc.Hierarchy(g, **opts).solve(b, tol=1e-8)
    res = {}
    for prec in (amg.AMG_PREC_FP64, amg.AMG_PREC_FP32):
        h = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, precision=prec, **opts)
        assert h.status == 0
        bd = cuda(b)
        xd = torch.zeros_like(bd)
        st, info, hist = h.solve(bd, xd, tol=1e-8)
        assert st == 0
        x = xd.cpu().numpy()
        res[prec] = (info.iterations, rel(x, ref.x), info.true_rel_residual,
                     resid_gap(orc, g, opts, x, ref.x) / np.linalg.norm(b))
        h.close()
    it64, e64, _, g64 = res[amg.AMG_PREC_FP64]
    it32, e32, t32, g32 = res[amg.AMG_PREC_FP32]
    print(f"rdiag2d_2048: oracle {ref.iterations} it; fp64 GPU {it64} it, rel err {e64:.2e}; "
          f"fp32-precond {it32} it, rel err {e32:.2e}, ||A(x-x_orc)||/||b|| {g32:.2e}, true res {t32:.2e}")
    assert abs(it64 - ref.iterations) <= 1 and e64 < 1e-7
    assert it32 <= it64 + 3 and g32 <= 2.1e-8
