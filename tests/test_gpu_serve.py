"""GPU checks of the continuous-batching server (amg_server_*).

* A request's result is the same alone and in the mix: requests solved one at
  a time (one slot) and the same requests submitted together to four slots,
  with graphs of uneven size in flight at once, give bit-identical solutions
  (every kernel is deterministic).
* Slots overlap (peak active > 1) and every solution meets its tolerance.
* Under a memory cap that holds only a few hierarchies, idle hierarchies are
  evicted and re-built and every request still completes.
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


def run(amg, graphs, reqs, max_active, cap=8 << 30, **opts):
    srv = amg.Server(cap, max_active, degree=4, passes=3, **opts)
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


@pytest.mark.parametrize("precision", [0, 1])
def test_same_result_alone_and_in_the_mix(amg, precision):
    graphs = pool()
    reqs = requests(graphs)
    alone, _ = run(amg, graphs, reqs, 1, precision=precision)
    mixed, stats = run(amg, graphs, reqs, 4, precision=precision)
    assert stats.peak_active > 1
    assert stats.completed == len(reqs)
    for (gi, b), (sa, xa, ia, _), (sm, xm, im, _) in zip(reqs, alone, mixed):
        assert sa == sm == amg.AMG_OK
        assert np.array_equal(xa, xm)
        assert ia.iterations == im.iterations
        A = sparse_laplacian(graphs[gi])
        assert np.linalg.norm(b - A @ xm) <= 1e-7 * np.linalg.norm(b)


def test_memory_cap_evicts_idle_hierarchies(amg):
    graphs = pool()
    reqs = requests(graphs, per=2)
    res, stats = run(amg, graphs, reqs, 2, cap=160 << 20)
    assert stats.evictions > 0 and stats.setups > len(graphs)
    for (gi, b), (st, x, info, lat) in zip(reqs, res):
        assert st == amg.AMG_OK
        A = sparse_laplacian(graphs[gi])
        assert np.linalg.norm(b - A @ x) <= 1e-7 * np.linalg.norm(b)
        assert lat > 0
