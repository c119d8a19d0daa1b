"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every symbol include/amg.h declares, validates arguments before
touching the device, reports the absence of a device as AMG_ERR_CUDA, and the
binding's structures match the header's layouts."""
import os
import re
import subprocess

import numpy as np
import pytest

import graphgen as gg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "amg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(amg_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def amg():
    import paper_1307_6305_gb300 as pkg

    pkg.lib()
    return pkg


def test_exports_every_declared_symbol(amg):
    declared = header_symbols()
    assert len(declared) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", amg.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (amg_\w+)", out))
    assert set(declared) <= exported, set(declared) - exported
    assert set(declared) == set(amg.SYMBOLS)
    for s in declared:
        assert hasattr(amg.lib(), s)


def test_default_options(amg):
    o = amg.amg_default_options()
    assert (o.degree, o.passes, o.coarse_max, o.max_levels, o.inner_iters, o.restart) == (4, 3, 64, 30, 2, 5)
    assert o.precision == amg.AMG_PREC_FP64 and o.lambda0_ratio == 0.1
    assert o.cycle == amg.AMG_CYCLE_K and o.amli_alpha == 0.25 and o.rho == 0.0
    assert o.aggregation == amg.AMG_AGG_MATCHING and o.mis_k == 4


def test_degree_for_matches_oracle(amg, orc):
    """amg_degree_for (library) and the oracle's reading of Eq. (bound-on-m)
    are separate implementations; they agree wherever m <= 16."""
    for ratio in (0.02, 0.05, 0.1, 0.2, 0.5):
        for rho in np.geomspace(1e-4, 2.0, 37):
            m = orc.degree_for(rho, ratio)
            want = m if 0 <= m <= 16 else -1
            assert amg.amg_degree_for(rho, ratio) == want, (rho, ratio)
    assert amg.amg_degree_for(1 / 3, 0.1) == 4
    for bad in ((0.0, 0.1), (-1.0, 0.1), (0.3, 0.0), (0.3, 1.0)):
        assert amg.amg_degree_for(*bad) == -1


def test_argument_errors_before_device(amg):
    g = gg.grid2d_5pt(4)
    rp, col, w = g.rowptr, g.col, g.w
    st, h = amg.amg_setup(0, rp, col, w)
    assert st == amg.AMG_ERR_INVALID_ARG and not h.value
    # row indices are 32-bit in the kernels: n above 2^31 - 2^16 is refused
    # before any buffer is read
    st, h = amg.amg_setup((1 << 31) - (1 << 16) + 1, rp, col, w)
    assert st == amg.AMG_ERR_INVALID_ARG and "2^31" in amg.amg_last_error(None)
    st, h = amg.amg_setup(g.n, None, col, w)
    assert st == amg.AMG_ERR_INVALID_ARG
    for bad in (dict(degree=-1), dict(degree=17), dict(passes=0), dict(inner_iters=9), dict(restart=0),
                dict(precision=3), dict(lambda0_ratio=1.5), dict(coarse_max=0), dict(cycle=2), dict(rho=-1.0),
                dict(rho=1e-12), dict(cycle=1, amli_alpha=0.0), dict(cycle=1, amli_alpha=0.1),
                dict(cycle=1, inner_iters=1), dict(aggregation=2), dict(aggregation=1, mis_k=0),
                dict(aggregation=1, mis_k=17), dict(passes=17), dict(coarse_max=4097), dict(max_levels=0),
                dict(max_levels=65), dict(inner_iters=0), dict(restart=17), dict(max_iters=-1),
                dict(precision=-1), dict(lambda0_ratio=0.0), dict(lambda0_ratio=float("nan")),
                dict(rho=float("inf")), dict(rho=float("nan")), dict(cycle=1, amli_alpha=1.0), dict(cycle=-1)):
        st, h = amg.amg_setup(g.n, rp, col, w, None, amg.amg_default_options(**bad))
        assert st == amg.AMG_ERR_INVALID_ARG, bad
        assert amg.amg_last_error(None)
    rp2 = rp.copy(); rp2[0] = 1
    st, h = amg.amg_setup(g.n, rp2, col, w)
    assert st == amg.AMG_ERR_INVALID_ARG
    st, h = amg.amg_setup(g.n, rp, col, w, None, None, 7)
    assert st == amg.AMG_ERR_INVALID_ARG
    assert amg.amg_solve(None, np.zeros(3), np.zeros(3), 1, 3, 1e-8) == amg.AMG_ERR_INVALID_ARG


def test_match_entry_points_refuse_null_pointers(amg):
    """amg_match and amg_match_noalloc check every pointer on the host before
    any device work (the addresses below are never dereferenced)."""
    fake = 1 << 20
    for fn in (amg.amg_match, amg.amg_match_noalloc):
        for col, s in ((None, fake), (fake, None), (None, None)):
            st, _, _ = fn(16, fake, col, s, 0, fake, fake)
            assert st == amg.AMG_ERR_INVALID_ARG, (fn.__name__, col, s)
            assert "non-NULL" in amg.amg_last_error(None)
        st, _, _ = fn(16, None, fake, fake, 0, fake, fake)
        assert st == amg.AMG_ERR_INVALID_ARG
        st, _, _ = fn(0, fake, fake, fake, 0, fake, fake)
        assert st == amg.AMG_ERR_INVALID_ARG


def test_option_limits_are_inclusive(amg):
    """Options at the documented limits pass validation: on a machine without
    a device, setup gets as far as the device check (AMG_ERR_CUDA)."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("checks the no-device path")
    g = gg.grid2d_5pt(4)
    for edge in (dict(degree=0), dict(degree=16), dict(passes=16), dict(coarse_max=1), dict(coarse_max=4096),
                 dict(max_levels=1), dict(max_levels=64), dict(inner_iters=8), dict(restart=1),
                 dict(restart=16), dict(max_iters=0), dict(aggregation=1, mis_k=1),
                 dict(aggregation=1, mis_k=16), dict(cycle=1, inner_iters=2, amli_alpha=0.25),
                 dict(rho=1 / 3), dict(precision=1)):
        st, h = amg.amg_setup(g.n, g.rowptr, g.col, g.w, None, amg.amg_default_options(**edge))
        assert st == amg.AMG_ERR_CUDA, (edge, st, amg.amg_last_error(None))


def test_no_device_is_reported(amg):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a device is present")
    g = gg.grid2d_5pt(4)
    st, h = amg.amg_setup(g.n, g.rowptr, g.col, g.w)
    assert st == amg.AMG_ERR_CUDA and not h.value
    assert "device" in amg.amg_last_error(None)


def test_server_argument_errors(amg):
    import ctypes as C

    cfg = amg.amg_server_config()
    cfg.mem_cap_bytes = 1 << 30
    cfg.max_active = 0
    cfg.opt = amg.amg_default_options()
    h = C.c_void_p()
    assert amg.lib().amg_server_create(C.byref(cfg), C.byref(h)) == amg.AMG_ERR_INVALID_ARG
    cfg.max_active = 2
    cfg.mem_cap_bytes = 10
    assert amg.lib().amg_server_create(C.byref(cfg), C.byref(h)) == amg.AMG_ERR_INVALID_ARG
    import torch

    if not torch.cuda.is_available():
        cfg.mem_cap_bytes = 1 << 30
        assert amg.lib().amg_server_create(C.byref(cfg), C.byref(h)) == amg.AMG_ERR_CUDA


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the field names, offsets and sizes
    of the C declarations (a C program built against include/amg.h reports
    them), so options and reports cross the boundary unchanged."""
    from helpers import assert_layouts_match, c_struct_layouts
    from paper_1307_6305_gb300 import binding as B

    structs = [("amg_options", B.amg_options), ("amg_info", B.amg_info),
               ("amg_server_config", B.amg_server_config), ("amg_server_stats_t", B.amg_server_stats_t)]
    layout = c_struct_layouts(os.path.join(ROOT, "include"), "amg.h", structs, tmp_path)
    if layout is None:
        pytest.skip("no C compiler")
    assert_layouts_match(layout, structs)
