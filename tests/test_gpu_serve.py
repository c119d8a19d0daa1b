"""GPU checks of the continuous-batching server (amg_server_*).

* A request's result is the same alone and in the mix: requests solved one at
  a time (one slot) and the same requests submitted together to four slots,
  with graphs of uneven size in flight at once.  With batching off
  (batch_max 1) requests for one graph take turns on the single-vector path
  and the solutions are bit-identical.  With batching on (batch_max 8) the
  queued requests of one graph are solved together in the block path (fewer
  solve calls than requests) while a lone request takes the single-vector
  path; both meet ||r|| <= 1e-8 ||b||, so a request's two results differ by a
  vector whose residual is at most 2e-8 ||b|| -- the bound checked -- and
  their iteration counts by at most a few.
* Slots overlap (peak active > 1) and every solution meets its tolerance.
* Under a memory cap that holds only a few hierarchies, idle hierarchies are
  evicted and re-built, resident bytes stay under the cap and every request
  still completes.
* A hierarchy larger than the cap fails its request with AMG_ERR_OOM instead
  of waiting forever; a non-finite right-hand side is refused at submission.
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


def pool():
    return [gg.random_geometric(20000, 51), gg.grid2d_5pt(150), gg.grid3d_7pt(30, 1.0),
            gg.random_geometric(60000, 52), gg.grid2d_random_diag(120, 7), gg.grid3d_7pt(18, None)]


def requests(graphs, per=3):
    out = []
    for r in range(per):
        for gi, g in enumerate(graphs):
            out.append((gi, gg.rhs(g.n, 1000 * gi + r, gg.is_pure_laplacian(g))))
    return out


def run(amg, graphs, reqs, max_active, cap=8 << 30, batch_max=8, **opts):
    srv = amg.Server(cap, max_active, batch_max=batch_max, degree=4, passes=3, **opts)
    ids = [srv.add_graph(g) for g in graphs]
    if max_active == 1:
        res = []
        for gi, b in reqs:
            res.append(srv.wait(srv.submit(ids[gi], b)))
    else:
        tickets = [srv.submit(ids[gi], b) for gi, b in reqs]
        res = [srv.wait(t) for t in tickets]
    stats = srv.stats()
    srv.close()
    return res, stats


@pytest.mark.parametrize("batch_max", [8, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_same_result_alone_and_in_the_mix(amg, precision, batch_max):
    graphs = pool()
    reqs = requests(graphs)
    alone, sa = run(amg, graphs, reqs, 1, batch_max=batch_max, precision=precision)
    mixed, stats = run(amg, graphs, reqs, 4, batch_max=batch_max, precision=precision)
    assert sa.solves == len(reqs)               # one at a time: no batches
    assert stats.peak_active > 1
    assert stats.completed == len(reqs)
    if batch_max > 1:
        assert stats.solves < len(reqs)         # same-graph requests shared a solve
    else:
        assert stats.solves == len(reqs)
    for (gi, b), (sa, xa, ia, _), (sm, xm, im, _) in zip(reqs, alone, mixed):
        assert sa == sm == amg.AMG_OK
        A = sparse_laplacian(graphs[gi])
        assert np.linalg.norm(b - A @ xm) <= 1e-7 * np.linalg.norm(b)
        assert im.rel_residual <= 1e-8 and ia.rel_residual <= 1e-8
        if batch_max == 1:
            assert np.array_equal(xa, xm)
            assert ia.iterations == im.iterations
        else:
            assert np.linalg.norm(A @ (xa - xm)) <= 2.1e-8 * np.linalg.norm(b)
            assert abs(ia.iterations - im.iterations) <= 3


def hierarchy_bytes(amg, graphs):
    """Arena bytes of each graph's hierarchy, read off the server's resident
    total while the graphs are set up one at a time under an ample cap."""
    srv = amg.Server(8 << 30, 1, degree=4, passes=3)
    out, before = [], 0
    for g in graphs:
        gid = srv.add_graph(g)
        assert srv.wait(srv.submit(gid, gg.rhs(g.n, 5, gg.is_pure_laplacian(g))))[0] == amg.AMG_OK
        now = srv.stats().resident_bytes
        out.append(now - before)
        before = now
    srv.close()
    return out


def test_memory_cap_evicts_idle_hierarchies(amg):
    graphs = pool()
    sizes = hierarchy_bytes(amg, graphs)
    cap = int(1.3 * max(sizes))
    assert cap < sum(sizes)          # not every hierarchy fits at once
    reqs = requests(graphs, per=2)
    res, stats = run(amg, graphs, reqs, 2, cap=cap)
    assert stats.peak_resident_bytes <= cap and stats.resident_bytes <= cap
    assert stats.evictions > 0 and stats.setups > len(graphs)
    for (gi, b), (st, x, info, lat) in zip(reqs, res):
        assert st == amg.AMG_OK
        A = sparse_laplacian(graphs[gi])
        assert np.linalg.norm(b - A @ x) <= 1e-7 * np.linalg.norm(b)
        assert lat > 0


def test_hierarchy_larger_than_cap_fails_cleanly(amg):
    g = gg.grid2d_5pt(150)
    srv = amg.Server(1 << 20, 2, degree=4, passes=3)
    gid = srv.add_graph(g)
    st, x, info, lat = srv.wait(srv.submit(gid, gg.rhs(g.n, 3, gg.is_pure_laplacian(g))))
    assert st == amg.AMG_ERR_OOM
    stats = srv.stats()
    assert stats.resident_bytes == 0 and stats.completed == 1
    srv.close()


def test_non_finite_rhs_is_refused_at_submission(amg):
    g = gg.grid2d_5pt(40)
    srv = amg.Server(1 << 30, 2, degree=4, passes=3)
    gid = srv.add_graph(g)
    b = gg.rhs(g.n, 3, True)
    for bad in (np.nan, np.inf):
        bb = b.copy()
        bb[7] = bad
        with pytest.raises(amg.AmgError) as e:
            srv.submit(gid, bb)
        assert e.value.status == amg.AMG_ERR_INVALID_ARG
    st, x, info, lat = srv.wait(srv.submit(gid, b))
    assert st == amg.AMG_OK and info.rel_residual <= 1e-8
    srv.close()
