"""GPU checks of the leaf kernel: the inner flexible-CG solve at the level just
above the dense two-level operator, run as one thread-block-cluster kernel
per call with its vectors in shared memory (AMG_GB300_LEAF=0 keeps the
multi-kernel path).

For hierarchies where the leaf engages (fewer launches per solve):
  * fp64: the same iteration count as the multi-kernel path, residual
    histories within 1e-10 of each other and of the oracle, solutions within
    1e-7 relative;
  * fp32 preconditioner: the same iteration count within 1, every solution
    meets the tolerance;
  * the degenerate settings the kernel branches on: degree 0 and 1, one and
    three inner steps, a pure Laplacian (d = 0), an irregular random graph;
  * each of the CTA sizes the kernel is built for (256, 512 and 1024 threads,
    AMG_GB300_LEAF_THREADS), whose row-to-lane assignment differs.
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


def solve(amg, g, b, monkeypatch, leaf, converge=True, nt=256, **opts):
    monkeypatch.setenv("AMG_GB300_LEAF", "1" if leaf else "0")
    monkeypatch.setenv("AMG_GB300_LEAF_THREADS", str(nt))
    h = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, **opts)
    assert h.status == 0, h.error
    x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    st, info, hist = h.solve(torch.as_tensor(b, device="cuda"), x, tol=1e-8)
    want = amg.AMG_OK if converge else amg.AMG_ERR_NOT_CONVERGED
    assert st == want, amg.amg_last_error(h.h)
    out = (x.cpu().numpy(), info.iterations, np.asarray(hist), h.launch_count(), h.n_levels)
    h.close()
    return out


CASES = {
    "grid3d_20": (lambda: gg.grid3d_7pt(20, 1.0), dict(degree=5, passes=3)),
    # degree 0 and 1 smoothers have E_m > 1 for kappa = 10 and need not
    # converge: 25 iterations are compared, the oracle decides the status
    "grid3d_20_deg0": (lambda: gg.grid3d_7pt(20, 1.0), dict(degree=0, passes=3, max_iters=25)),
    "grid3d_20_deg1": (lambda: gg.grid3d_7pt(20, 1.0), dict(degree=1, passes=3, max_iters=25)),
    "grid3d_20_nu1": (lambda: gg.grid3d_7pt(20, 1.0), dict(degree=3, passes=3, inner_iters=1)),
    "grid3d_20_nu3": (lambda: gg.grid3d_7pt(20, 1.0), dict(degree=3, passes=3, inner_iters=3)),
    "grid3d_18_pure": (lambda: gg.grid3d_7pt(18, None), dict(degree=4, passes=3)),
    "rdiag_90": (lambda: gg.grid2d_random_diag(90, 5), dict(degree=4, passes=3)),
    "random_4000": (lambda: random_graph(4000, 0.0015, 11, wmax=5, d_frac=0.02), dict(degree=4, passes=2)),
}


@pytest.mark.parametrize("nt", [256, 512, 1024])
@pytest.mark.parametrize("name", sorted(CASES))
def test_leaf_matches_multikernel_and_oracle(amg, orc, name, nt, monkeypatch):
    make, opts = CASES[name]
    g = make()
    b = gg.rhs(g.n, 31, gg.is_pure_laplacian(g))
    ref = orc.Hierarchy(g, **opts).solve(b, tol=1e-8)
    conv = ref.status == 0
    x1, it1, h1, n1, L = solve(amg, g, b, monkeypatch, True, conv, nt, **opts)
    x0, it0, h0, n0, _ = solve(amg, g, b, monkeypatch, False, conv, **opts)
    assert L >= 4, "hierarchy too shallow for the leaf level"
    assert n1 < n0, f"leaf kernel not used ({n1} vs {n0} launches)"
    assert it1 == it0
    # absolute 1e-10 on relative residuals, relative where a non-converging
    # history grows above 1
    assert (np.abs(h1 - h0) <= 1e-10 * np.maximum(1.0, np.abs(h0))).all()
    m = min(len(h1), len(ref.history))
    assert (np.abs(h1[:m] - ref.history[:m]) <= 1e-10 * np.maximum(1.0, np.abs(ref.history[:m]))).all()
    if not conv:
        return
    scale = np.abs(x0).max()
    assert np.abs(x1 - x0).max() <= 1e-7 * scale
    assert abs(it1 - ref.iterations) <= 1
    A = sparse_laplacian(g)
    assert np.linalg.norm(b - A @ x1) <= 1e-7 * np.linalg.norm(b)


@pytest.mark.parametrize("nt", [256, 512, 1024])
@pytest.mark.parametrize("name", ["grid3d_20", "grid3d_18_pure", "random_4000"])
def test_leaf_fp32(amg, name, nt, monkeypatch):
    make, opts = CASES[name]
    g = make()
    b = gg.rhs(g.n, 32, gg.is_pure_laplacian(g))
    x1, it1, _, n1, _ = solve(amg, g, b, monkeypatch, True, nt=nt, precision=amg.AMG_PREC_FP32, **opts)
    x0, it0, _, n0, _ = solve(amg, g, b, monkeypatch, False, precision=amg.AMG_PREC_FP32, **opts)
    assert n1 < n0
    assert abs(it1 - it0) <= 1
    A = sparse_laplacian(g)
    for x in (x0, x1):
        assert np.linalg.norm(b - A @ x) <= 1e-7 * np.linalg.norm(b)
    assert np.linalg.norm(A @ (x1 - x0)) <= 2.1e-8 * np.linalg.norm(b)


def test_leaf_repeatable(amg, monkeypatch):
    """Two solves of the same system give bit-identical results (the cluster
    reductions fold partials in a fixed order)."""
    make, opts = CASES["random_4000"]
    g = make()
    b = gg.rhs(g.n, 33, False)
    xa, ita, ha, _, _ = solve(amg, g, b, monkeypatch, True, **opts)
    xb, itb, hb, _, _ = solve(amg, g, b, monkeypatch, True, **opts)
    assert ita == itb
    assert np.array_equal(xa, xb) and np.array_equal(ha, hb)
