"""GPU checks of the batched (multi right-hand side) solve.

All right-hand sides of one amg_solve call are solved together with block
kernels (SpMM forms of every operator) and per-column Krylov scalars.  Each
column must give the solution of its own single solve:
  * fp64: per column the oracle's iterations +-1, column 0's residual history
    within 1e-10 of the oracle's, solutions within 1e-7 relative;
  * fp32 preconditioner: every column reaches 1e-8 (fp64 outer residual) and
    the gap to the oracle's solution has residual <= 2e-8 ||b||.
"""
import json
import os

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


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def rhs_block(g, seeds):
    return np.stack([gg.rhs(g.n, s, gg.is_pure_laplacian(g)) for s in seeds])  # row j = column j


@pytest.mark.parametrize("nrhs", [2, 5, 32, 40])
def test_fp64_batch_matches_oracle_per_column(amg, orc, nrhs):
    g = gg.grid3d_7pt(16, 1.0)
    opts = dict(degree=5, passes=3)
    B = rhs_block(g, range(100, 100 + nrhs))
    h = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, **opts)
    assert h.status == 0
    Bd = torch.as_tensor(B, device="cuda")
    Xd = torch.zeros_like(Bd)
    st, info, hist = h.solve(Bd, Xd, tol=1e-8, nrhs=nrhs, ld=g.n)
    assert st == amg.AMG_OK, amg.amg_last_error(h.h)
    X = Xd.cpu().numpy()
    oh = orc.Hierarchy(g, **opts)
    its = []
    for j in range(nrhs):
        ref = oh.solve(B[j], tol=1e-8)
        its.append(ref.iterations)
        assert rel(X[j], ref.x) < 1e-7, j
        if j == 0:
            m = min(len(hist), len(ref.history))
            assert np.abs(hist[:m] - ref.history[:m]).max() <= 1e-10
    assert abs(info.iterations - max(its)) <= 1
    assert info.true_rel_residual < 1e-7


def test_pure_laplacian_batch_and_host_buffers(amg, orc):
    g = gg.grid2d_random_diag(40, 3)
    opts = dict(degree=4, passes=3)
    B = rhs_block(g, range(7, 10))
    h = amg.Hierarchy.from_graph(g, **opts)                # host graph
    X = np.zeros_like(B)
    st, info, hist = h.solve(B, X, tol=1e-8, nrhs=3, ld=g.n)  # host vectors
    assert st == amg.AMG_OK
    oh = orc.Hierarchy(g, **opts)
    for j in range(3):
        ref = oh.solve(B[j], tol=1e-8)
        assert rel(X[j], ref.x) < 1e-7
        assert abs(X[j].mean()) < 1e-12


@pytest.mark.parametrize("nrhs", [8, 32])
def test_fp32_batch(amg, orc, nrhs):
    g = gg.grid3d_7pt(24, 1.0)
    opts = dict(degree=5, passes=3)
    B = rhs_block(g, range(4000, 4000 + nrhs))
    h = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, precision=amg.AMG_PREC_FP32, **opts)
    Bd = torch.as_tensor(B, device="cuda")
    Xd = torch.zeros_like(Bd)
    st, info, hist = h.solve(Bd, Xd, tol=1e-8, nrhs=nrhs, ld=g.n)
    assert st == amg.AMG_OK
    X = Xd.cpu().numpy()
    A = sparse_laplacian(g)
    oh = orc.Hierarchy(g, **opts)
    for j in (0, nrhs // 2, nrhs - 1):
        ref = oh.solve(B[j], tol=1e-8)
        assert info.iterations <= ref.iterations + 3
        assert np.linalg.norm(A @ (X[j] - ref.x)) <= 2.1e-8 * np.linalg.norm(B[j])
    for j in range(nrhs):
        assert np.linalg.norm(B[j] - A @ X[j]) <= 1e-7 * np.linalg.norm(B[j])


def test_tuning_cache_file(amg, tmp_path):
    g = gg.grid3d_7pt(12, 1.0)
    cache = tmp_path / "tune.json"
    old = os.environ.get("AMG_GB300_TUNE_CACHE")
    os.environ["AMG_GB300_TUNE_CACHE"] = str(cache)
    try:
        B = torch.as_tensor(rhs_block(g, range(32)), device="cuda")
        X = torch.zeros_like(B)
        h = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, degree=5, passes=3)
        assert h.solve(B, X, tol=1e-8, nrhs=32, ld=g.n)[0] == amg.AMG_OK
        entries = json.loads(cache.read_text())
        assert len(entries) == 1
        (kb, tile), = entries.values()
        assert kb in (8, 16, 32) and tile in (128, 256, 512)
        X2 = torch.zeros_like(B)
        h2 = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, degree=5, passes=3, hash_salt=1)
        assert h2.solve(B, X2, tol=1e-8, nrhs=32, ld=g.n)[0] == amg.AMG_OK
        assert len(json.loads(cache.read_text())) == 1       # same shape: decision reused, not re-tuned
    finally:
        if old is None:
            os.environ.pop("AMG_GB300_TUNE_CACHE", None)
        else:
            os.environ["AMG_GB300_TUNE_CACHE"] = old


@pytest.mark.slow
def test_full_size_grid3d_96_32rhs_fp32(amg, orc):
    """The batching workload at full size: 96^3 7-point Laplacian with d = 1 on
    the boundary, 32 right-hand sides (seeds 4000..4031), degree 5, fp32
    preconditioner / fp64 flexible CG, solved in one batched call."""
    g, p = gg.workload("grid3d_96x32")
    B = rhs_block(g, p["rhs_seeds"])
    h = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, precision=amg.AMG_PREC_FP32,
                                 degree=p["degree"], passes=p["passes"])
    Bd = torch.as_tensor(B, device="cuda")
    Xd = torch.zeros_like(Bd)
    st, info, hist = h.solve(Bd, Xd, tol=1e-8, nrhs=32, ld=g.n)
    assert st == amg.AMG_OK
    X = Xd.cpu().numpy()
    A = sparse_laplacian(g)
    oh = orc.Hierarchy(g, degree=p["degree"], passes=p["passes"])
    for j in (0, 31):
        ref = oh.solve(B[j], tol=1e-8)
        assert np.linalg.norm(A @ (X[j] - ref.x)) <= 2.1e-8 * np.linalg.norm(B[j])
    worst = max(np.linalg.norm(B[j] - A @ X[j]) / np.linalg.norm(B[j]) for j in range(32))
    print(f"grid3d_96x32 batched fp32: {info.iterations} iterations, worst true residual {worst:.2e}, "
          f"solve {info.solve_ms:.1f} ms")
    assert worst <= 1e-7
