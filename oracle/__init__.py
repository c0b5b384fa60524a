"""FP64 CPU oracle for the timing hot path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it.

``tdp_oracle.c`` holds the arithmetic (plain single-threaded C, double
precision); this module compiles it on first use and wraps it with ctypes.
Each function cites the passage of the paper it restates.

Parity unpinned: none of the functions here.  Every function is pinned by the
CPU tests (hand-computed circuits, brute-force path enumeration, invariants,
finite differences); see ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tdp_oracle.c")
_LIB = os.path.join(_HERE, "libtdp_oracle.so")
_lib = None

OR_OK, OR_ERR_INVALID, OR_ERR_CYCLE, OR_ERR_OOM = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Paths(C.Structure):
    _fields_ = [("n_paths", C.c_int64), ("n_pins_total", C.c_int64), ("n_viol", C.c_int32),
                ("viol", C.POINTER(C.c_int32)), ("ep", C.POINTER(C.c_int32)),
                ("rank", C.POINTER(C.c_int32)), ("slack", C.POINTER(C.c_double)),
                ("pin_ptr", C.POINTER(C.c_int64)), ("pins", C.POINTER(C.c_int32))]


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.c_void_p
        lib.or_sta.restype = C.c_int
        lib.or_sta.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P, P, P, P, P,
                               C.c_double, C.c_double, C.c_double, P, P, C.c_double,
                               P, P, P, P, P, P, P, P, P]
        lib.or_topk.restype = C.c_int
        lib.or_topk.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P, P, P, P, C.c_double,
                                C.c_int, C.c_int, C.c_int, P, C.c_int, C.POINTER(_Paths)]
        lib.or_free_paths.restype = None
        lib.or_free_paths.argtypes = [C.POINTER(_Paths)]
        lib.or_update_pairs.restype = C.c_int
        lib.or_update_pairs.argtypes = [C.c_int, P, C.c_int64, P, P, P, C.c_double,
                                        C.c_double, C.c_double, P, P]
        lib.or_loss.restype = C.c_double
        lib.or_loss.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P, P, P, P, P, P, P,
                                C.c_double, C.c_int, P, P]
        lib.or_net_weights.restype = C.c_int
        lib.or_net_weights.argtypes = [C.c_int, P, P, C.c_double, C.c_double, C.c_double, P]
        lib.or_loss_kind.restype = C.c_double
        lib.or_loss_kind.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P, P, P, P, P, P, P,
                                     C.c_double, C.c_int, C.c_int, P, P]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def sta(nl, x=None, y=None, T: float = 0.0) -> dict:
    """Static timing analysis in FP64 (Section II-B, Eqs. (2)-(4), Eq. (8)).

    Returns per-pin ``tnet, arr, req, slack, pred`` and per-net ``cload, dnet``
    (delay of the net's driver cell), plus scalars ``wns, tns``.
    """
    lib = _load()
    x = _f64(nl.x if x is None else x)
    y = _f64(nl.y if y is None else y)
    pc, npt, ct = _i32(nl.pin_cell), _i32(nl.net_ptr), _i32(nl.cell_type)
    dx, dy, cap, rd = _f64(nl.pin_dx), _f64(nl.pin_dy), _f64(nl.pin_cap), _f64(nl.cell_rdrv)
    n = nl.n_pins
    out = {k: np.zeros(n) for k in ("tnet", "arr", "req", "slack")}
    out["cload"] = np.zeros(nl.n_nets)
    out["dnet"] = np.zeros(nl.n_nets)
    out["pred"] = np.zeros(n, dtype=np.int32)
    wns, tns = C.c_double(), C.c_double()
    st = lib.or_sta(nl.n_cells, n, nl.n_nets, _p(pc), _p(npt), _p(ct), _p(dx), _p(dy), _p(cap),
                    _p(rd), nl.r_per_um, nl.c_per_um, nl.d0_ps, _p(x), _p(y), float(T),
                    _p(out["tnet"]), _p(out["cload"]), _p(out["dnet"]), _p(out["arr"]),
                    _p(out["req"]), _p(out["slack"]), _p(out["pred"]), C.byref(wns),
                    C.byref(tns))
    if st != OR_OK:
        raise RuntimeError(f"oracle sta failed with status {st}")
    out["wns"], out["tns"], out["T"] = wns.value, tns.value, float(T)
    return out


def clock_period(nl, factor: float, x=None, y=None) -> float:
    """Clock period = factor x the largest endpoint arrival at this placement.

    With T = 0 every endpoint violates and WNS = -(largest endpoint arrival).
    """
    return factor * (-sta(nl, x, y, 0.0)["wns"])


def topk(nl, timing: dict, n_endpoints: int = -1, K: int = 1, keep_nonneg: bool = False,
         endpoints=None) -> dict:
    """report_timing_endpoint(n, K) of Section III-B on the FP64 timing.

    Returns the violating endpoints sorted by (slack, pin) and, per path,
    ``ep, rank, slack`` and its pins (startpoint first) as ``pin_ptr/pins``.
    ``endpoints`` (optional) restricts the search to the given endpoint pins.
    """
    lib = _load()
    pc, npt, ct = _i32(nl.pin_cell), _i32(nl.net_ptr), _i32(nl.cell_type)
    res = _Paths()
    if endpoints is None:
        epl, n_list = np.zeros(1, dtype=np.int32), -1
    else:
        epl = _i32(endpoints)
        n_list = len(epl)
    st = lib.or_topk(nl.n_cells, nl.n_pins, nl.n_nets, _p(pc), _p(npt), _p(ct),
                     _p(_f64(timing["tnet"])), _p(_f64(timing["dnet"])),
                     _p(_f64(timing["arr"])), float(timing["T"]), int(n_endpoints), int(K),
                     int(bool(keep_nonneg)), _p(epl), int(n_list), C.byref(res))
    if st != OR_OK:
        raise RuntimeError(f"oracle topk failed with status {st}")
    n, m, nv = res.n_paths, res.n_pins_total, res.n_viol
    out = {
        "viol": np.ctypeslib.as_array(res.viol, (max(nv, 1),))[:nv].copy() if nv else np.zeros(0, np.int32),
        "ep": np.ctypeslib.as_array(res.ep, (max(n, 1),))[:n].copy(),
        "rank": np.ctypeslib.as_array(res.rank, (max(n, 1),))[:n].copy(),
        "slack": np.ctypeslib.as_array(res.slack, (max(n, 1),))[:n].copy(),
        "pin_ptr": np.ctypeslib.as_array(res.pin_ptr, (n + 1,)).copy(),
        "pins": np.ctypeslib.as_array(res.pins, (max(m, 1),))[:m].copy(),
    }
    lib.or_free_paths(C.byref(res))
    return out


# cell types of the netlist interface
_FF, _PO = 1, 3


def report_timing(nl, timing: dict, n: int, keep_nonneg: bool = False) -> dict:
    """report_timing(n) as Section III-B describes OpenTimer's command (the
    one Table I measures): take the n endpoints of lowest slack, the n
    lowest-slack paths of each, and report the n paths of lowest slack among
    those n x n, worst first.

    Without ``keep_nonneg`` only failing endpoints and paths of negative slack
    take part.  Equal slacks are ordered as in ``topk``, by the pin sequence
    read from the endpoint: by endpoint pin, then by rank at the endpoint.
    Returns ``ep, rank, slack, pin_ptr, pins`` of the reported paths.
    """
    n = int(n)
    if n < 0:
        raise ValueError("report_timing: n < 0")
    ct = np.asarray(nl.cell_type)[np.asarray(nl.pin_cell)]
    eps = np.nonzero((np.asarray(nl.pin_dir) == 0) & ((ct == _FF) | (ct == _PO)))[0]
    es = timing["T"] - np.asarray(timing["arr"])[eps]
    if not keep_nonneg:
        eps, es = eps[es < 0.0], es[es < 0.0]
    worst = eps[np.lexsort((eps, es))][:n]
    empty = {"ep": np.zeros(0, np.int32), "rank": np.zeros(0, np.int32), "slack": np.zeros(0),
             "pin_ptr": np.zeros(1, np.int64), "pins": np.zeros(0, np.int32)}
    if n == 0 or len(worst) == 0:
        return empty
    P = topk(nl, timing, -1, n, keep_nonneg, endpoints=worst)
    sel = np.lexsort((P["rank"], P["ep"], P["slack"]))[:n]
    lens = np.diff(P["pin_ptr"])[sel]
    ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    pins = np.concatenate([P["pins"][P["pin_ptr"][k]:P["pin_ptr"][k + 1]] for k in sel]) if len(sel) \
        else np.zeros(0, np.int32)
    return {"ep": P["ep"][sel], "rank": P["rank"][sel], "slack": P["slack"][sel], "pin_ptr": ptr,
            "pins": pins.astype(np.int32)}


def update_pairs(nl, paths: dict, wns: float, w0: float, w1: float, in_p=None, w=None):
    """Eq. (w_ij): update the persistent pin-pair set P (by sink pin) and weights."""
    lib = _load()
    in_p = np.zeros(nl.n_pins, dtype=np.uint8) if in_p is None else in_p.astype(np.uint8).copy()
    w = np.zeros(nl.n_pins) if w is None else _f64(w).copy()
    pd = np.ascontiguousarray(nl.pin_dir, dtype=np.uint8)
    n = len(paths["slack"])
    st = lib.or_update_pairs(nl.n_pins, _p(pd), n, _p(_f64(paths["slack"])),
                             _p(np.ascontiguousarray(paths["pin_ptr"], dtype=np.int64)),
                             _p(_i32(paths["pins"])), float(wns), float(w0), float(w1),
                             _p(in_p), _p(w))
    if st != OR_OK:
        raise RuntimeError(f"oracle update_pairs failed with status {st}")
    return in_p, w


LOSS_KINDS = {"quadratic": 0, "hpwl": 1, "euclid": 2}


def loss(nl, in_p, w, beta: float = 1.0, x=None, y=None, drop_fixed: bool = True,
         kind: str = "quadratic"):
    """PP = beta * sum_{(i,j) in P} w_ij Q(i,j) (Eq. (9)); returns (PP, gx, gy).

    kind "hpwl" / "euclid" replaces Q(i,j) by the pair's HPWL or linear
    Euclidean distance (the ablation of Section IV)."""
    lib = _load()
    x = _f64(nl.x if x is None else x)
    y = _f64(nl.y if y is None else y)
    gx = np.zeros(nl.n_cells)
    gy = np.zeros(nl.n_cells)
    pp = lib.or_loss_kind(nl.n_cells, nl.n_pins, nl.n_nets, _p(_i32(nl.pin_cell)), _p(_i32(nl.net_ptr)),
                          _p(_f64(nl.pin_dx)), _p(_f64(nl.pin_dy)),
                          _p(np.ascontiguousarray(nl.cell_fixed, dtype=np.uint8)), _p(x), _p(y),
                          _p(np.ascontiguousarray(in_p, dtype=np.uint8)), _p(_f64(w)), float(beta),
                          int(bool(drop_fixed)), LOSS_KINDS[kind], _p(gx), _p(gy))
    return float(pp), gx, gy


def net_weights(nl, timing: dict, alpha: float, gamma: float, w=None):
    """Net weights from pin slacks with momentum: the net-weighting baseline
    of Section II-C and of the "w/o Path Extraction" ablation (Section IV),
    under this reading (the paper gives no formula): s_e = worst pin slack of
    net e, c_e = min(1, max(0, -s_e) / |WNS|) (0 if WNS = 0),
    w_e <- alpha w_e + (1 - alpha)(1 + gamma c_e), w starting at 1.
    Returns (new weights, number of nets with s_e < 0)."""
    lib = _load()
    w = np.ones(nl.n_nets) if w is None else _f64(w).copy()
    n = lib.or_net_weights(nl.n_nets, _p(_i32(nl.net_ptr)), _p(_f64(timing["slack"])), float(timing["wns"]),
                           float(alpha), float(gamma), _p(w))
    return w, int(n)
