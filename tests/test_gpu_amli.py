"""GPU parity of the stationary AMLI W-cycle (cycle = AMG_CYCLE_AMLI) and of
the automatic smoother degree (rho > 0, Eq. bound-on-m) against the oracle.

* one application of the cycle at level 0 (amg_apply_kcycle applies the
  handle's cycle) within 1e-11 of the oracle's AMLI cycle, relative to the
  result's max norm;
* the preconditioned solve: residual history within 1e-10 of the oracle's,
  iterations within 1, solution within 1e-7 relative;
* fp32 preconditioner: converges to 1e-8 with the solution's error against the
  fp64 oracle solution bounded like the K-cycle's;
* several right-hand sides in one call are solved column by column and equal
  the single solves.
"""
import numpy as np
import pytest

import graphgen as gg
from helpers import random_graph, sparse_laplacian

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


CASES = {
    "grid2d_64": (lambda: gg.grid2d_5pt(64), dict(degree=3, passes=2)),
    "grid3d_20_d": (lambda: gg.grid3d_7pt(20, 1.0), dict(degree=5, passes=3)),
    "rdiag_48": (lambda: gg.grid2d_random_diag(48, 3), dict(degree=4, passes=3)),
    "rand_w": (lambda: random_graph(1500, 0.004, 5, wmax=4, d_frac=0.05), dict(degree=4, passes=2)),
    "nu3": (lambda: gg.grid3d_7pt(16, 1.0), dict(degree=4, passes=3, inner_iters=3, amli_alpha=0.15)),
    "rho": (lambda: gg.grid3d_7pt(18, None), dict(rho=0.1, passes=3)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_amli_matches_oracle(amg, orc, name):
    make, opts = CASES[name]
    g = make()
    gh = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, cycle=amg.AMG_CYCLE_AMLI, **opts)
    assert gh.status == 0, gh.error
    oh = orc.Hierarchy(g, cycle=1, **opts)
    assert oh.status == 0
    assert gh.n_levels == oh.n_levels
    # one cycle application at level 0
    r = gg.rhs(g.n, 5, gg.is_pure_laplacian(g))
    out = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    gh.apply("kcycle", 0, cuda(r), out)
    ref = oh.amli_cycle(0, r)
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-11 * np.abs(ref).max()
    # the solve
    b = gg.rhs(g.n, 17, gg.is_pure_laplacian(g))
    x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    st, info, hist = gh.solve(cuda(b), x, tol=1e-8)
    assert st == amg.AMG_OK, amg.amg_last_error(gh.h)
    res = oh.solve(b, tol=1e-8)
    assert res.status == 0
    assert abs(info.iterations - res.iterations) <= 1
    m = min(len(hist), len(res.history))
    assert np.abs(hist[:m] - res.history[:m]).max() <= 1e-10
    xs = x.cpu().numpy()
    assert np.abs(xs - res.x).max() <= 1e-7 * np.abs(res.x).max()


@pytest.mark.parametrize("name", ["grid3d_20_d", "rand_w"])
def test_amli_fp32(amg, orc, name):
    make, opts = CASES[name]
    g = make()
    gh = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, cycle=amg.AMG_CYCLE_AMLI,
                                  precision=amg.AMG_PREC_FP32, **opts)
    b = gg.rhs(g.n, 18, gg.is_pure_laplacian(g))
    x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    st, info, _ = gh.solve(cuda(b), x, tol=1e-8)
    assert st == amg.AMG_OK
    res = orc.Hierarchy(g, cycle=1, **opts).solve(b, tol=1e-8)
    assert info.iterations <= res.iterations + 3
    A = sparse_laplacian(g)
    xs = x.cpu().numpy()
    assert np.linalg.norm(b - A @ xs) <= 1e-7 * np.linalg.norm(b)
    assert np.linalg.norm(A @ (xs - res.x)) <= 2.1e-8 * np.linalg.norm(b)


def test_amli_several_rhs_column_by_column(amg):
    make, opts = CASES["grid3d_20_d"]
    g = make()
    B = np.stack([gg.rhs(g.n, s, False) for s in (40, 41, 42)])
    gh = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, cycle=amg.AMG_CYCLE_AMLI, **opts)
    X = torch.zeros(3, g.n, dtype=torch.float64, device="cuda")
    st, info, _ = gh.solve(cuda(B), X, tol=1e-8, nrhs=3, ld=g.n)
    assert st == amg.AMG_OK
    for j in range(3):
        x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
        assert gh.solve(cuda(B[j]), x, tol=1e-8)[0] == amg.AMG_OK
        assert torch.equal(x, X[j])


def test_rho_sets_degree_like_the_oracle(amg, orc):
    g = gg.grid3d_7pt(14, 1.0)
    gh = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, rho=0.05, passes=3)
    oh = orc.Hierarchy(g, rho=0.05, passes=3)
    m = amg.amg_degree_for(0.05, 0.1)
    assert m == oh.opts.degree
    lam0, lam1, coef = gh.level_smoother(0)
    assert len(coef) == m + 1
    b = gg.rhs(g.n, 19, False)
    x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    st, info, hist = gh.solve(cuda(b), x, tol=1e-8)
    res = oh.solve(b, tol=1e-8)
    assert st == amg.AMG_OK and abs(info.iterations - res.iterations) <= 1
    k = min(len(hist), len(res.history))
    assert np.abs(hist[:k] - res.history[:k]).max() <= 1e-10
