"""Failure handling made on the host, checked on the GPU.

* Injected allocation failure: with AMG_GB300_FAIL_ALLOC=k the k-th device
  allocation of amg_setup fails as if the pool were exhausted.  Walking k over
  every allocation of a small setup, each attempt must return AMG_ERR_OOM with
  the injected message and leave the process usable; once k exceeds the
  allocation count the setup succeeds, and a solve on that handle matches the
  oracle.  Nothing faults the GPU: the failure is a status returned by the
  host-side allocator.
* Non-finite right-hand sides (NaN, +-inf, or a norm that overflows fp64) are
  refused with AMG_ERR_INVALID_ARG instead of returning an iterate built from
  garbage, for one and for several right-hand sides, host and device buffers;
  the handle then solves a valid right-hand side normally.
"""
import os

import numpy as np
import pytest

import graphgen as gg

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


@pytest.mark.parametrize("name,make,opts", [
    ("grid2d_24", lambda: gg.grid2d_5pt(24), dict(degree=3, passes=2)),
    ("grid3d_12_d", lambda: gg.grid3d_7pt(12, 1.0), dict(degree=5, passes=3, precision=1)),
])
def test_every_setup_allocation_failure_is_reported(amg, orc, name, make, opts):
    g = make()
    old = os.environ.get("AMG_GB300_FAIL_ALLOC")
    k, failures = 1, 0
    try:
        while True:
            os.environ["AMG_GB300_FAIL_ALLOC"] = str(k)
            h = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, **opts)
            if h.status == amg.AMG_OK:
                break
            assert h.status == amg.AMG_ERR_OOM, (k, h.status, h.error)
            assert "injected allocation failure" in h.error, (k, h.error)
            failures += 1
            k += 1
            assert k < 5000, "the setup makes more allocations than expected"
    finally:
        if old is None:
            os.environ.pop("AMG_GB300_FAIL_ALLOC", None)
        else:
            os.environ["AMG_GB300_FAIL_ALLOC"] = old
    assert failures >= 20, failures          # the walk covered a real setup
    torch.cuda.synchronize()
    # the handle that survived the walk and a fresh one both solve normally
    fresh = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, **opts)
    assert fresh.status == amg.AMG_OK, fresh.error
    b = gg.rhs(g.n, 3, gg.is_pure_laplacian(g))
    ref = orc.Hierarchy(g, **{k2: v for k2, v in opts.items() if k2 != "precision"}).solve(b, tol=1e-8)
    for hh in (h, fresh):
        bd = cuda(b)
        xd = torch.zeros_like(bd)
        st, info, hist = hh.solve(bd, xd, tol=1e-8)
        assert st == amg.AMG_OK and hist[-1] <= 1e-8
        if "precision" not in opts:
            assert abs(info.iterations - ref.iterations) <= 1
            assert np.abs(xd.cpu().numpy() - ref.x).max() <= 1e-7 * np.abs(ref.x).max()
    h.close()
    fresh.close()


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf, 1e300])
@pytest.mark.parametrize("where", ["device", "host"])
def test_non_finite_rhs_is_refused(amg, bad, where):
    g = gg.grid3d_7pt(16, 1.0)
    h = amg.Hierarchy.from_graph(g, mem_space=amg.AMG_MEM_DEVICE, degree=5, passes=3)
    assert h.status == amg.AMG_OK
    b = gg.rhs(g.n, 11, False)
    bb = b.copy()
    bb[g.n // 3] = bad
    if bad == 1e300:
        bb[g.n // 2] = bad                      # ||b||^2 overflows
    mk = cuda if where == "device" else (lambda a: np.ascontiguousarray(a, np.float64))
    x = torch.zeros(g.n, dtype=torch.float64, device="cuda") if where == "device" else np.zeros(g.n)
    st, info, hist = h.solve(mk(bb), x, tol=1e-8)
    assert st == amg.AMG_ERR_INVALID_ARG, st
    assert "non-finite" in amg.amg_last_error(h.h)
    # several right-hand sides, one of them bad
    B = np.concatenate([b, bb, b])
    X = torch.zeros(3 * g.n, dtype=torch.float64, device="cuda") if where == "device" else np.zeros(3 * g.n)
    st, info, hist = h.solve(mk(B), X, tol=1e-8, nrhs=3)
    assert st == amg.AMG_ERR_INVALID_ARG, st
    # the handle still solves a valid right-hand side
    x2 = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    st, info, hist = h.solve(cuda(b), x2, tol=1e-8)
    assert st == amg.AMG_OK and hist[-1] <= 1e-8
    h.close()
