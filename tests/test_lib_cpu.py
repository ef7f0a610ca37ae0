"""Host-side checks of libww.so that need no GPU: it loads, exports every entry
point include/ww.h declares, rejects bad arguments before touching the device,
and its FP64 cost-table builder agrees with the oracle's tables."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2609_36267_b300 as ww

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "ww.h")).read()
    return sorted(set(re.findall(r"\b(ww_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = ww.lib()
    syms = header_symbols()
    assert len(syms) >= 16
    for s in syms:
        assert hasattr(lib, s), s


def test_status_strings_and_defaults():
    assert ww.status_string(0) == "ok"
    assert "infeasible" in ww.status_string(-4)
    p = ww.default_params()
    assert p.box_half_width == 2 and p.steep_cap_ppm == 30000 and abs(p.steep_rad - 1.0) < 1e-7


def test_argument_checks_without_device():
    lib = ww.lib()
    g = ctypes.c_void_p()
    assert lib.ww_build_lut(1.0, ctypes.byref(g)) == ww.WW_ERR_INVALID_ARG  # needs L > 1
    assert lib.ww_build_lut(float("nan"), ctypes.byref(g)) == ww.WW_ERR_INVALID_ARG
    assert lib.ww_residues(None, 0, None, None, 10, 10, None, None, None) == ww.WW_ERR_INVALID_ARG
    dummy = ctypes.c_void_p(16)
    # grids must be at least 2 x 2
    assert lib.ww_residues(dummy, 0, None, None, 1, 10, dummy, dummy, None) == ww.WW_ERR_INVALID_ARG
    assert lib.ww_integrate(dummy, 0, None, None, dummy, 5, 1, dummy, dummy, None) == ww.WW_ERR_INVALID_ARG
    bad = ww.default_params(box_half_width=7)
    assert lib.ww_solve_mcf(dummy, dummy, dummy, 4, 4, ctypes.byref(bad), None, dummy, dummy, dummy, dummy,
                            None) == ww.WW_ERR_INVALID_ARG
    assert lib.ww_workspace_bytes(1, 5) == -1
    assert lib.ww_workspace_bytes(8192, 9000) > 8192 * 9000 * 20


def test_server_refuses_a_budget_below_one_request():
    """Every device allocation of a server counts against its budget: a budget
    that cannot hold one request of the largest accepted size is refused before
    anything is allocated."""
    cfg = ww.ServerConfig(2 << 20, 1 << 24, 4)
    h = ctypes.c_void_p()
    prm = ww.default_params()
    assert ww.lib().ww_server_create(ctypes.byref(cfg), ctypes.byref(prm), ctypes.byref(h)) == ww.WW_ERR_INVALID_ARG
    assert not h.value


def test_lut_from_table_roundtrip():
    t = (np.arange(128 * 256) % 30000).astype(np.int16).reshape(128, 256)
    lut = ww.Lut.from_table(9.0, t)
    assert np.array_equal(lut.table(), t)
    with pytest.raises(ww.WWError):
        lut.cost100()  # only built tables carry FP64 values


# Agreement of the library's FP64 table builder with the oracle's tables: the
# int16 tables are identical entrywise at every L (no entry is excused), and
# 100*c agrees to 3e-7 relative (100*c + 1 scale).  The oracle's values are in
# turn pinned to an independent quadrature (tests/test_oracle_lut_chain.py).
REL_TOL = 3e-7


@pytest.mark.parametrize("L", [4.0, 6.0, 9.0, 16.0, 50.0])
def test_library_lut_matches_oracle(L):
    path = os.path.join(GOLDEN, f"lut_oracle_L{L:g}.npz")
    z = np.load(path)
    co, to = z["cost100"], z["table"]
    lut = ww.Lut.build(L)
    c, t = lut.cost100(), lut.table()
    fin = np.isfinite(co) & (co < 32767)
    assert np.array_equal(np.isfinite(c), np.isfinite(co))
    d = np.abs(c - co)[fin] / (co[fin] + 1.0)
    assert d.max() <= REL_TOL, d.max()
    assert np.array_equal(t, to)
    # the fp32 100 ln(P0/P+) tables of the interpolated lookup: the same FP64
    # agreement, then one rounding each
    r, ro = lut.ratio100(), z["ratio100"]
    assert np.all(np.abs(r.astype(np.float64) - ro) <= REL_TOL * (np.abs(ro) + 1.0) + np.spacing(np.abs(ro)))
    # the cache hands out the same table
    assert np.array_equal(ww.Lut.build(L).table(), t)
