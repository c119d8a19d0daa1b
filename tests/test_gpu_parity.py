"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bar (see the tolerance notes in the library's design document):
  * integer/index work bit-exact: per-level sizes, aggregate maps, coarse CSR
    (pattern and values: all test weights are integers, so every Galerkin sum
    is exact), lambda1;
  * single fp64 operations (SpMV, smoother, transfers, coarsest solve, one
    K-cycle) within 1e-11 of the oracle relative to the result's max norm
    (different FMA contraction/summation order only);
  * outer residual history |h_gpu(k) - h_orc(k)| <= 1e-10 (h = ||r_k||/||b||),
    iteration counts within +-1, final solutions within 1e-7 relative.
"""
import numpy as np
import pytest

import graphgen as gg
from helpers import complete_graph, path_graph, random_graph, star_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def amg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1307_6305_gb300 as pkg

    pkg.lib()
    return pkg


def cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def pair(amg, orc, g, mem=None, **opts):
    mem = amg.AMG_MEM_DEVICE if mem is None else mem
    gh = amg.Hierarchy.from_graph(g, mem_space=mem, **opts)
    assert gh.status == 0, gh.error
    ok = {k: v for k, v in opts.items() if k != "precision"}
    oh = orc.Hierarchy(g, **ok)
    assert oh.status == 0
    return gh, oh


def close(a, b, rtol):
    a = np.asarray(a)
    b = np.asarray(b)
    scale = max(np.abs(b).max(), 1e-300)
    err = np.abs(a - b).max() / scale
    assert err <= rtol, f"max rel err {err:.3e} > {rtol:.1e}"


GRAPHS = {
    "grid2d_64": (lambda: gg.grid2d_5pt(64), dict(degree=3, passes=2)),
    "grid3d_20_d": (lambda: gg.grid3d_7pt(20, 1.0), dict(degree=5, passes=3)),
    "rdiag_48": (lambda: gg.grid2d_random_diag(48, 3), dict(degree=4, passes=3)),
    "rand_w": (lambda: random_graph(700, 0.006, 3, wmax=4, d_frac=0.05), dict(degree=4, passes=2)),
    "delaunay_14": (lambda: gg.delaunay3d(14, 5), dict(degree=4, passes=3)),
    "rgg_3000": (lambda: gg.random_geometric(3000, 5), dict(degree=4, passes=3)),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_hierarchy_bit_exact(amg, orc, name):
    make, opts = GRAPHS[name]
    g = make()
    gh, oh = pair(amg, orc, g, **opts)
    assert gh.n_levels == oh.n_levels
    for k in range(oh.n_levels):
        assert gh.level_n(k) == oh.level_n(k)
        for a, b in zip(gh.level_csr(k), oh.level_csr(k)):
            assert np.array_equal(a, b), (name, k)
        if k + 1 < oh.n_levels:
            assert np.array_equal(gh.level_agg(k), oh.level_agg(k))
            l0, l1, coef = gh.level_smoother(k)
            ol0, ol1 = oh.level_lambda(k)
            assert l1 == ol1 and l0 == ol0
            close(coef, oh.level_cheb(k), 1e-12)


def test_host_and_device_inputs_agree(amg, orc):
    g = gg.grid3d_7pt(12, 1.0)
    a = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_HOST, degree=5, passes=3)
    b = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, degree=5, passes=3)
    assert a.status == b.status == 0
    assert a.n_levels == b.n_levels
    for k in range(a.n_levels - 1):
        assert np.array_equal(a.level_agg(k), b.level_agg(k))


@pytest.mark.parametrize("name", ["grid2d_64", "grid3d_20_d", "rand_w"])
def test_level_operations(amg, orc, name):
    make, opts = GRAPHS[name]
    g = make()
    gh, oh = pair(amg, orc, g, **opts)
    L = oh.n_levels
    for k in range(L):
        n = oh.level_n(k)
        v = gg.uniform_pm1(100 + k, n)
        vd = cuda(v)
        out = torch.zeros_like(vd)
        gh.apply("spmv", k, vd, out)
        close(out.cpu().numpy(), oh.spmv(k, v), 1e-13)
        out.zero_()
        gh.apply("kcycle", k, vd, out)
        close(out.cpu().numpy(), oh.kcycle(k, v), 1e-11)
        if k + 1 < L:
            out.zero_()
            gh.apply("smoother", k, vd, out)
            close(out.cpu().numpy(), oh.smooth(k, v), 1e-12)
            nH = oh.level_n(k + 1)
            rH = torch.zeros(nH, dtype=torch.float64, device="cuda")
            gh.apply("restrict", k, vd, rH)
            close(rH.cpu().numpy(), oh.restrict(k, v), 1e-14)
            e = gg.uniform_pm1(200 + k, nH)
            x = cuda(v)
            gh.apply("prolong_add", k, cuda(e), x)
            close(x.cpu().numpy(), oh.prolong_add(k, e, v), 1e-15)
        else:
            out.zero_()
            gh.coarse_solve(vd, out)
            close(out.cpu().numpy(), oh.coarse_solve(v), 1e-11)


@pytest.mark.parametrize("name", list(GRAPHS))
def test_solve_matches_oracle(amg, orc, name):
    make, opts = GRAPHS[name]
    g = make()
    gh, oh = pair(amg, orc, g, **opts)
    b = gg.rhs(g.n, 7, gg.is_pure_laplacian(g))
    ref = oh.solve(b, tol=1e-8)
    assert ref.status == 0
    bd = cuda(b)
    xd = torch.zeros_like(bd)
    st, info, hist = gh.solve(bd, xd, tol=1e-8)
    assert st == amg.AMG_OK
    assert abs(info.iterations - ref.iterations) <= 1
    m = min(len(hist), len(ref.history))
    assert np.abs(hist[:m] - ref.history[:m]).max() <= 1e-10
    close(xd.cpu().numpy(), ref.x, 1e-7)
    assert info.true_rel_residual < 1e-7
    assert info.n_levels == ref.n_levels
    assert info.grid_complexity == pytest.approx(ref.grid_complexity, rel=1e-12)
    assert info.op_complexity == pytest.approx(ref.op_complexity, rel=1e-12)


def test_host_vectors_and_multiple_rhs(amg, orc):
    g = gg.grid3d_7pt(10, 1.0)
    gh, oh = pair(amg, orc, g, degree=5, passes=3)
    B = np.stack([gg.rhs(g.n, s, False) for s in (1, 2, 3)])        # row j = rhs j
    X = np.zeros_like(B)
    st, info, hist = gh.solve(B, X, tol=1e-8, nrhs=3, ld=g.n)
    assert st == amg.AMG_OK
    for j in range(3):
        ref = oh.solve(B[j], tol=1e-8)
        close(X[j], ref.x, 1e-7)


def test_matching_pass_bit_exact(amg, orc):
    for seed in range(8):
        g = random_graph(400, 0.01, seed, wmax=3)
        s = g.w.astype(np.float64)
        mate_o, agg_o, nH_o, rounds_o = orc.match(g.rowptr, g.col, s, 31 * seed)
        mate = torch.zeros(g.n, dtype=torch.int32, device="cuda")
        agg = torch.zeros_like(mate)
        st, nH, rounds = amg.amg_match(g.n, cuda(g.rowptr, torch.int64), cuda(g.col, torch.int32), cuda(s),
                                       31 * seed, mate, agg)
        assert st == 0
        assert np.array_equal(mate.cpu().numpy(), mate_o)
        assert np.array_equal(agg.cpu().numpy(), agg_o)
        assert nH == nH_o and rounds == rounds_o


def _bad(g, **kw):
    return gg.Graph(g.n, kw.get("rowptr", g.rowptr), kw.get("col", g.col), kw.get("w", g.w), kw.get("d", g.d))


def test_validation_codes_match_oracle(amg, orc):
    g = gg.grid2d_5pt(5)
    cases = []
    w = g.w.copy(); w[3] = 2.0; cases.append(_bad(g, w=w))
    cases.append(_bad(g, w=-g.w))
    w = g.w.copy(); w[5] = np.nan; cases.append(_bad(g, w=w))
    col = g.col.copy(); col[0] = 0; cases.append(_bad(g, col=col))
    col = g.col.copy(); col[0] = 99; cases.append(_bad(g, col=col))
    col = g.col.copy(); col[[0, 1]] = col[[1, 0]]; cases.append(_bad(g, col=col))
    rp = g.rowptr.copy(); rp[2] = rp[1] - 1; cases.append(_bad(g, rowptr=rp))
    d = np.zeros(g.n); d[1] = -1; cases.append(_bad(g, d=d))
    cases.append(gg.csr_from_edges(6, np.array([0, 1, 3, 4]), np.array([1, 2, 4, 5])))
    cases.append(gg.csr_from_edges(6, np.array([0, 1, 3, 4]), np.array([1, 2, 4, 5]), d=np.array([1.0, 0, 0, 0, 0, 0])))
    cases.append(gg.csr_from_edges(6, np.array([0, 1, 3, 4]), np.array([1, 2, 4, 5]), d=np.array([1.0, 0, 0, 0, 0, 2.0])))
    for c in cases:
        ref = orc.Hierarchy(c).status
        for mem in (amg.AMG_MEM_HOST, amg.AMG_MEM_DEVICE):
            gh = amg.Hierarchy.from_graph(c, mem_space=mem)
            assert gh.status == ref, (gh.status, ref, gh.error)


@pytest.mark.parametrize("make,opts", [
    (lambda: gg.csr_from_edges(1, np.zeros(0, np.int64), np.zeros(0, np.int64)), {}),
    (lambda: path_graph(2), {}),
    (lambda: path_graph(300), dict(degree=3, passes=2, coarse_max=4)),
    (lambda: complete_graph(90), dict(degree=3, passes=2, coarse_max=8)),
    (lambda: star_graph(200), dict(coarse_max=8)),
    (lambda: gg.grid2d_5pt(20), dict(coarse_max=4096)),
    # degree 0 is not a convergent smoother (E_0 = 4.5 > 1): compare a capped run
    (lambda: gg.grid2d_5pt(33), dict(degree=0, passes=1, max_iters=25)),
    (lambda: gg.grid3d_7pt(7, 1.0), dict(degree=1, passes=1, inner_iters=1, restart=1)),
    (lambda: gg.grid3d_7pt(9, 1.0), dict(degree=6, passes=4, inner_iters=3, restart=8)),
])
def test_edge_cases_match_oracle(amg, orc, make, opts):
    g = make()
    gh, oh = pair(amg, orc, g, **opts)
    b = gg.rhs(g.n, 11, gg.is_pure_laplacian(g))
    ref = oh.solve(b, tol=1e-8)
    bd = cuda(b)
    xd = torch.zeros_like(bd)
    st, info, hist = gh.solve(bd, xd, tol=1e-8)
    assert st == ref.status
    assert abs(info.iterations - ref.iterations) <= 1
    m = min(len(hist), len(ref.history))
    assert np.abs(hist[:m] - ref.history[:m]).max() <= 1e-10
    if np.abs(ref.x).max() > 0:
        close(xd.cpu().numpy(), ref.x, 1e-7)
    else:
        assert np.abs(xd.cpu().numpy()).max() == 0


@pytest.mark.slow
def test_full_size_grid3d_128(amg, orc):
    """The benchmark workload at full size: 128^3 7-point Laplacian with d = 1 on
    the boundary faces, degree 5, three matching passes per level."""
    g, p = gg.workload("grid3d_128")
    gh, oh = pair(amg, orc, g, degree=p["degree"], passes=p["passes"])
    assert gh.n_levels == oh.n_levels
    for k in range(oh.n_levels - 1):
        assert np.array_equal(gh.level_agg(k), oh.level_agg(k))
    b = gg.rhs(g.n, p["rhs_seeds"][0], False)
    ref = oh.solve(b, tol=1e-8)
    bd = cuda(b)
    xd = torch.zeros_like(bd)
    st, info, hist = gh.solve(bd, xd, tol=1e-8)
    assert st == 0 and abs(info.iterations - ref.iterations) <= 1
    m = min(len(hist), len(ref.history))
    assert np.abs(hist[:m] - ref.history[:m]).max() <= 1e-10
    close(xd.cpu().numpy(), ref.x, 1e-7)


@pytest.mark.parametrize("precision", [0, 1])
def test_split_rows_match_one_thread_per_row(amg, orc, precision, monkeypatch):
    """Small levels run their SELL kernels with several warps per 32-row slice
    (AMG_GB300_SPLIT=0 turns that off).  Both forms solve the same problem:
    the same iteration count, residual histories within 1e-10 (fp64) and
    solutions within 1e-7; and the split form still meets the oracle."""
    g = gg.grid3d_7pt(24, 1.0)
    opts = dict(degree=5, passes=3, precision=precision)
    b = gg.rhs(g.n, 77, False)
    runs = {}
    for flag in ("0", "1"):
        monkeypatch.setenv("AMG_GB300_SPLIT", flag)
        h = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, **opts)
        x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
        st, info, hist = h.solve(cuda(b), x, tol=1e-8)
        assert st == amg.AMG_OK
        runs[flag] = (x.cpu().numpy(), info.iterations, np.asarray(hist))
        h.close()
    (x0, i0, h0), (x1, i1, h1) = runs["0"], runs["1"]
    assert i0 == i1
    if precision == 0:
        assert np.abs(h0 - h1).max() <= 1e-10
        ref = orc.Hierarchy(g, degree=5, passes=3).solve(b, tol=1e-8)
        assert abs(i1 - ref.iterations) <= 1
        m = min(len(h1), len(ref.history))
        assert np.abs(h1[:m] - ref.history[:m]).max() <= 1e-10
    close(x1, x0, 1e-7)


@pytest.mark.parametrize("precision,cycle", [(0, 0), (1, 0), (0, 1)])
def test_split_prolongation_equals_fused(amg, monkeypatch, precision, cycle):
    """Levels of one warp per slice and >= 2^17 rows write x = u + P e_H with
    a streaming kernel and then run the residual on x; the fused kernel forms
    the same x_j inside the residual's gather.  Both do the same operations in
    the same order, so residual histories and solutions are equal bit for bit
    (AMG_GB300_PROLONG_SPLIT=0 selects the fused form on every level)."""
    g = gg.grid3d_7pt(64, 1.0)
    b = gg.rhs(g.n, 12, False)
    runs = []
    for split in ("1", "0"):
        monkeypatch.setenv("AMG_GB300_PROLONG_SPLIT", split)
        gh = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, degree=5, passes=3,
                                      precision=precision, cycle=cycle)
        assert gh.status == 0, gh.error
        assert gh.level_n(0) >= 1 << 17
        x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
        st, info, hist = gh.solve(cuda(b), x, tol=1e-8)
        assert st == amg.AMG_OK, amg.amg_last_error(gh.h)
        runs.append((hist, x.cpu().numpy(), gh.launch_count(), info.iterations))
        gh.close()
    (hs, xs, ls, its), (hf, xf, lf, itf) = runs
    assert its == itf
    assert np.array_equal(hs, hf) and np.array_equal(xs, xf)
    assert ls > lf          # the split form ran (one more launch per level-0 cycle)


@pytest.mark.parametrize("precision,cycle", [(0, 0), (1, 0), (0, 1)])
def test_column_offsets_equal_full_columns(amg, monkeypatch, precision, cycle):
    """Levels of >= 2^17 rows whose every |j - i| fits 16 bits store their
    columns also as offsets from the row, and the one-row-per-thread kernels
    read those; the same entries are summed in the same order, so residual
    histories and solutions equal those of the 32-bit columns bit for bit
    (AMG_GB300_DELTA=0 keeps 32-bit columns everywhere).  The smoother step's
    byte count (2 or 4 bytes per column) shows which layout ran."""
    g = gg.grid3d_7pt(64, 1.0)
    b = gg.rhs(g.n, 13, False)
    runs = []
    for delta in ("1", "0"):
        monkeypatch.setenv("AMG_GB300_DELTA", delta)
        gh = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, degree=5, passes=3,
                                      precision=precision, cycle=cycle)
        assert gh.status == 0, gh.error
        assert gh.level_n(0) >= 1 << 17
        gh.kernel_timing(True)
        x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
        st, info, hist = gh.solve(cuda(b), x, tol=1e-8)
        assert st == amg.AMG_OK, amg.amg_last_error(gh.h)
        launches, _, bytes_per_launch = gh.kernel_timing_read()
        assert launches > 0
        runs.append((hist, x.cpu().numpy(), info.iterations, bytes_per_launch))
        gh.close()
    (h1, x1, i1, b1), (h0, x0, i0, b0) = runs
    nnz = g.col.size  # stored off-diagonals of level 0
    assert b0 - b1 == pytest.approx(2.0 * nnz)
    assert i1 == i0
    assert np.array_equal(h1, h0) and np.array_equal(x1, x0)


@pytest.mark.parametrize("opts", [
    dict(degree=4, passes=3, lambda0_ratio=0.05),
    dict(degree=4, passes=3, hash_salt=0x9E3779B97F4A7C15),
    dict(degree=3, passes=2, lambda0_ratio=0.2, hash_salt=12345, coarse_max=32, restart=3),
])
def test_non_default_options_match_oracle(amg, orc, opts):
    """Options other than the benchmark's: the smoother interval ratio (Sec. 3)
    and the salt of the matching's tie-break hash (Sec. 2) reach both sides the
    same way -- aggregates bit for bit, smoother intervals and coefficients to
    rounding, and the solve's residual history within 1e-10."""
    g = random_graph(6000, 0.0012, 13, wmax=4, d_frac=0.02)
    gh, oh = pair(amg, orc, g, **opts)
    assert gh.n_levels == oh.n_levels
    for k in range(oh.n_levels - 1):
        assert np.array_equal(gh.level_agg(k), oh.level_agg(k))
        l0, l1, coef = gh.level_smoother(k)
        o0, o1 = oh.level_lambda(k)
        assert l1 == o1 and l0 == pytest.approx(o0, rel=1e-15)
        ref = oh.level_cheb(k)
        assert np.abs(coef - ref).max() <= 1e-12 * np.abs(ref).max()
    b = gg.rhs(g.n, 43, False)
    res = oh.solve(b, tol=1e-8)
    x = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    st, info, hist = gh.solve(cuda(b), x, tol=1e-8)
    assert st == res.status and abs(info.iterations - res.iterations) <= 1
    m = min(len(hist), len(res.history))
    assert np.abs(hist[:m] - res.history[:m]).max() <= 1e-10
    close(x.cpu().numpy(), res.x, 1e-7)
