"""GPU parity of aggregation by a maximal independent set of the graph of A^k
(aggregation = AMG_AGG_MIS, Sec. 2 steps (A)-(B)) against the oracle.

* bit-exact: level sizes, aggregate maps of every level, coarse operators
  (pattern and values: integer weights make every Galerkin sum exact);
* the solve with either cycle: residual histories within 1e-10, iterations
  within 1, solutions within 1e-7 relative;
* fp32 preconditioner: converges, solution error against the fp64 oracle
  bounded like the matching hierarchies'.
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
    "grid3d_24_pure_k4": (lambda: gg.grid3d_7pt(24, None), dict(degree=4, mis_k=4)),
    "grid3d_20_d_k2": (lambda: gg.grid3d_7pt(20, 1.0), dict(degree=5, mis_k=2)),
    "grid2d_96_k4": (lambda: gg.grid2d_5pt(96), dict(degree=4, mis_k=4)),
    "rand_k3": (lambda: random_graph(3000, 0.002, 8, wmax=5, d_frac=0.02), dict(degree=4, mis_k=3)),
    "rgg_k4": (lambda: gg.random_geometric(20000, 61), dict(degree=4, mis_k=4)),
    "delaunay_16_k2": (lambda: gg.delaunay3d(16, 5), dict(degree=4, mis_k=2)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_mis_hierarchy_bit_exact(amg, orc, name):
    make, opts = CASES[name]
    g = make()
    gh = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, aggregation=amg.AMG_AGG_MIS, **opts)
    assert gh.status == 0, gh.error
    oh = orc.Hierarchy(g, aggregation=1, **opts)
    assert gh.n_levels == oh.n_levels
    for k in range(gh.n_levels):
        assert gh.level_n(k) == oh.level_n(k)
        grp, gcol, gval, gdiag = gh.level_csr(k)[:4]
        orp, ocol, oval, odiag = oh.level_csr(k)[:4]
        assert np.array_equal(grp, orp) and np.array_equal(gcol, ocol)
        assert np.array_equal(gval, oval) and np.array_equal(gdiag, odiag)
        if k + 1 < gh.n_levels:
            assert np.array_equal(gh.level_agg(k), oh.level_agg(k))


@pytest.mark.parametrize("cycle", [0, 1])
@pytest.mark.parametrize("name", ["grid3d_24_pure_k4", "rand_k3", "rgg_k4", "delaunay_16_k2"])
def test_mis_solve_matches_oracle(amg, orc, name, cycle):
    make, opts = CASES[name]
    g = make()
    gh = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, aggregation=amg.AMG_AGG_MIS, cycle=cycle,
                                  **opts)
    b = gg.rhs(g.n, 23, gg.is_pure_laplacian(g))
    x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    st, info, hist = gh.solve(cuda(b), x, tol=1e-8)
    assert st == amg.AMG_OK, amg.amg_last_error(gh.h)
    ref = orc.Hierarchy(g, aggregation=1, cycle=cycle, **opts).solve(b, tol=1e-8)
    assert ref.status == 0
    assert abs(info.iterations - ref.iterations) <= 1
    m = min(len(hist), len(ref.history))
    assert np.abs(hist[:m] - ref.history[:m]).max() <= 1e-10
    xs = x.cpu().numpy()
    assert np.abs(xs - ref.x).max() <= 1e-7 * np.abs(ref.x).max()


def test_mis_fp32(amg, orc):
    make, opts = CASES["grid3d_24_pure_k4"]
    g = make()
    gh = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, aggregation=amg.AMG_AGG_MIS,
                                  precision=amg.AMG_PREC_FP32, **opts)
    b = gg.rhs(g.n, 24, True)
    x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    st, info, _ = gh.solve(cuda(b), x, tol=1e-8)
    assert st == amg.AMG_OK
    ref = orc.Hierarchy(g, aggregation=1, **opts).solve(b, tol=1e-8)
    assert info.iterations <= ref.iterations + 3
    A = sparse_laplacian(g)
    xs = x.cpu().numpy()
    assert np.linalg.norm(b - A @ xs) <= 1e-7 * np.linalg.norm(b)
    assert np.linalg.norm(A @ (xs - ref.x)) <= 2.1e-8 * np.linalg.norm(b)
