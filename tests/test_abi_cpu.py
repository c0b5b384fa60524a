"""C-ABI checks that need no GPU.

* the shared library loads and exports every entry point ``include/tdp.h``
  declares (and the Python binding declares the same list);
* ``sta_build`` rejects malformed netlists on the host (cycles, dangling
  pins, nets without sinks, bad pin directions, bad cell pin counts,
  non-finite values) before touching the device;
* NULL handles return TDP_ERR_INVALID; nothing aborts across the boundary.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

import netgen
from paper_2503_11674_b300 import _abi
from paper_2503_11674_b300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return _abi.load()


def _declared():
    with open(os.path.join(ROOT, "include", "tdp.h")) as f:
        text = f.read()
    # declarations start a line with TDP_API (the macro's own definition does not)
    return sorted(set(re.findall(r"^TDP_API\s+[\w\s\*]*?\b(\w+)\s*\(", text, flags=re.M)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 15
    assert sorted(_abi.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n


def _build(lib, nl, prec=_abi.TDP_FP32):
    keep = [np.ascontiguousarray(a) for a in (nl.pin_cell.astype(np.int32), nl.net_ptr.astype(np.int32),
                                              nl.pin_dir.astype(np.uint8), nl.cell_type.astype(np.int32),
                                              nl.pin_dx.astype(np.float32), nl.pin_dy.astype(np.float32),
                                              nl.pin_cap.astype(np.float32), nl.cell_rdrv.astype(np.float32),
                                              nl.cell_fixed.astype(np.uint8))]
    desc = _abi.NetlistDesc(nl.n_cells, nl.n_pins, nl.n_nets, *[k.ctypes.data for k in keep],
                            nl.r_per_um, nl.c_per_um, nl.d0_ps)
    h = C.c_void_p()
    st = lib.sta_build(C.byref(desc), prec, None, C.byref(h))
    return st, h


def _cycle_netlist():
    # two inverters feeding each other, plus a PI/PO so that every net has a sink
    cells = [{"type": "COMB", "x": 0, "y": 0, "rdrv": 1}, {"type": "COMB", "x": 5, "y": 0, "rdrv": 1},
             {"type": "PO", "x": 9, "y": 0}]
    nets = [[(0, 1.0), (1, 1.0), (2, 1.0)], [(1, 1.0), (0, 1.0)]]
    return netgen.from_lists(cells, nets)


def test_cycle_is_rejected(lib):
    st, h = _build(lib, _cycle_netlist())
    assert st == _abi.TDP_ERR_CYCLE and not h.value
    assert b"loop" in lib.tdp_last_error()


@pytest.mark.parametrize("breaker", ["pin_dir", "pin_cell", "net_ptr", "cap_nan", "po_two_inputs",
                                     "comb_no_output", "precision"])
def test_malformed_netlists_are_rejected(lib, breaker):
    from golden_util import load
    _, nl = load("reconverge_tie")
    prec = _abi.TDP_FP32
    if breaker == "pin_dir":
        nl.pin_dir = nl.pin_dir.copy()
        nl.pin_dir[1] = 1
    elif breaker == "pin_cell":
        nl.pin_cell = nl.pin_cell.copy()
        nl.pin_cell[2] = 99
    elif breaker == "net_ptr":
        nl.net_ptr = nl.net_ptr.copy()
        nl.net_ptr[2] = nl.net_ptr[1] + 1          # a net with only its driver
    elif breaker == "cap_nan":
        nl.pin_cap = nl.pin_cap.copy()
        nl.pin_cap[4] = np.nan
    elif breaker == "po_two_inputs":
        nl.pin_cell = nl.pin_cell.copy()
        nl.pin_cell[6] = 4                         # G3.b moved onto the PO
    elif breaker == "comb_no_output":
        nl.cell_type = nl.cell_type.copy()
        nl.cell_type[4] = netgen.COMB              # the PO becomes a gate with no output
    elif breaker == "precision":
        prec = 7
    st, h = _build(lib, nl, prec)
    assert st == _abi.TDP_ERR_INVALID and not h.value
    assert len(lib.tdp_last_error()) > 0


def test_null_handles(lib):
    assert lib.sta_propagate(None, None, None, 0.0, None, None) == _abi.TDP_ERR_INVALID
    assert lib.extract_critical_paths(None, -1, 4, 0, None) == _abi.TDP_ERR_INVALID
    assert lib.attraction_update_pairs(None, 10.0, 0.2, None) == _abi.TDP_ERR_INVALID
    assert lib.attraction_loss_fwd(None, None, None, 1.0, None) == _abi.TDP_ERR_INVALID
    assert lib.attraction_loss_bwd(None, None, None, 1.0, None, None, None) == _abi.TDP_ERR_INVALID
    assert lib.sta_get_paths(None, None, None, None, None, None) == _abi.TDP_ERR_INVALID
    assert lib.report_timing(None, 10, 0, None) == _abi.TDP_ERR_INVALID
    assert lib.sta_join(None) == _abi.TDP_ERR_INVALID
    assert lib.sta_propagate_incremental(None, None, None, 0.0, None, None) == _abi.TDP_ERR_INVALID
    assert lib.sta_incremental_stats(None, None) == _abi.TDP_ERR_INVALID
    assert lib.attraction_set_loss_kind(None, 0) == _abi.TDP_ERR_INVALID
    lib.sta_destroy(None)
    h = C.c_void_p()
    assert lib.sta_build(None, 0, None, C.byref(h)) == _abi.TDP_ERR_INVALID


def test_debug_hooks_check_their_arguments_on_the_host(lib):
    """The failure-injection hooks reject bad arguments without touching a device."""
    n = C.c_int64(-7)
    assert lib.tdp_debug_fail_alloc(-1) == _abi.TDP_ERR_INVALID
    assert lib.tdp_debug_fail_alloc(3) == _abi.TDP_OK
    assert lib.tdp_debug_pending_alloc_failure(C.byref(n)) == _abi.TDP_OK and n.value == 3
    assert lib.tdp_debug_fail_alloc(0) == _abi.TDP_OK
    assert lib.tdp_debug_pending_alloc_failure(C.byref(n)) == _abi.TDP_OK and n.value == 0
    assert lib.tdp_debug_pending_alloc_failure(None) == _abi.TDP_ERR_INVALID
    assert lib.tdp_debug_set_sync_status(None, 1) == _abi.TDP_ERR_INVALID
