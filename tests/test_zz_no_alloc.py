"""amg_match_noalloc against amg_match.

amg_match_noalloc serves callers that may not allocate device memory (their
memory is owned by another allocator, or cudaFree's device-wide sync would
break their pipeline): its scratch is a fixed array inside the library.  It
must give exactly the matching amg_match gives (integer outputs: bit-exact),
call after call, since consecutive calls reuse the same scratch.  This file
is collected last so that a failing run that stops at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import graphgen as gg
from helpers import random_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def amg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1307_6305_gb300 as pkg

    pkg.lib()
    return pkg


def dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def run(fn, g, s, salt):
    mate = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
    agg = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
    st, nH, rounds = fn(g.n, dev(g.rowptr, torch.int64), dev(g.col, torch.int32), dev(s, torch.float64),
                        salt, mate, agg)
    return st, mate.cpu().numpy(), agg.cpu().numpy(), nH, rounds


def test_noalloc_matches_amg_match_on_consecutive_calls(amg):
    cases = [(random_graph(3000, 0.002, 1, wmax=3), 17), (gg.grid3d_7pt(40, None), 5),
             (gg.random_geometric(20000, 9), 0)]
    for g, salt in cases:                      # consecutive calls share the scratch
        s = g.w.astype(np.float64)
        ref = run(amg.amg_match, g, s, salt)
        got = run(amg.amg_match_noalloc, g, s, salt)
        assert ref[0] == amg.AMG_OK and got[0] == amg.AMG_OK, amg.amg_last_error(None)
        assert np.array_equal(got[1], ref[1])
        assert np.array_equal(got[2], ref[2])
        assert got[3] == ref[3] and got[4] == ref[4]
        assert got[3] < g.n


def test_noalloc_at_its_capacity_matches_amg_match_and_the_oracle(amg, orc):
    """The two-level scan of the coarse ids at its fixed limit: n = 2^20
    (1024^2 grid: 512 scan tiles, the full width of the block-sum scan) and
    n = 101^3 = 1,030,301 (a ragged last tile), twice in a row; integer
    outputs bit for bit against amg_match and against the oracle's matching."""
    for g, salt in ((gg.grid2d_5pt(1024), 3), (gg.grid3d_7pt(101, None), 11)):
        s = g.w.astype(np.float64)
        o_mate, o_agg, o_nH, o_rounds = orc.match(g.rowptr, g.col, s, salt)
        ref = run(amg.amg_match, g, s, salt)
        assert ref[0] == amg.AMG_OK, amg.amg_last_error(None)
        for _ in range(2):
            got = run(amg.amg_match_noalloc, g, s, salt)
            assert got[0] == amg.AMG_OK, amg.amg_last_error(None)
            assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])
            assert got[3] == ref[3] and got[4] == ref[4]
            assert np.array_equal(got[1], o_mate) and np.array_equal(got[2], o_agg)
            assert got[3] == o_nH and got[4] == o_rounds


def test_noalloc_rejects_sizes_beyond_capacity(amg):
    n = (1 << 20) + 1
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.ones(1, dtype=torch.float64, device="cuda")
    mate = torch.zeros(n, dtype=torch.int32, device="cuda")
    agg = torch.zeros(n, dtype=torch.int32, device="cuda")
    st, _, _ = amg.amg_match_noalloc(n, rp, col, s, 0, mate, agg)
    assert st == amg.AMG_ERR_INVALID_ARG
    assert "capacity" in amg.amg_last_error(None)
