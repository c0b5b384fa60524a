"""Python binding of the timing hot path (same names as the C ABI).

PyTorch supplies device memory and streams only; every step runs in the CUDA
library behind ``include/tdp.h``.  ``TimingGraph`` owns one ``tdp_graph``;
its methods are one-line calls into the ABI:

    sta_propagate            Section II-B, Eqs. (2)-(4), Eq. (8)
    extract_critical_paths   Section III-B, report_timing_endpoint(n, K)
    attraction_update_pairs  Section III-D, Eq. (w_ij)
    attraction_loss_fwd/bwd  Eq. (9), PP of Section III-D

``AttractionLoss`` is the ``torch.autograd.Function`` whose backward is the
hand-written adjoint kernel (``attraction_loss_bwd``).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _abi


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class TimingGraph:
    """One netlist on one GPU, in FP32 (``torch.float32``) or FP64."""

    def __init__(self, netlist, precision: str = "fp32", device: str | torch.device = "cuda",
                 stream: torch.cuda.Stream | None = None):
        self.lib = _abi.load()
        self.device = torch.device(device)
        if self.device.type != "cuda":
            raise ValueError("TimingGraph runs on a CUDA device only")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.dtype = {"fp32": torch.float32, "fp64": torch.float64}[precision]
        self.n_cells, self.n_pins, self.n_nets = netlist.n_cells, netlist.n_pins, netlist.n_nets
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        keep = {
            "pin_cell": _np(netlist.pin_cell, np.int32), "net_ptr": _np(netlist.net_ptr, np.int32),
            "pin_dir": _np(netlist.pin_dir, np.uint8), "cell_type": _np(netlist.cell_type, np.int32),
            "pin_dx": _np(netlist.pin_dx, np.float32), "pin_dy": _np(netlist.pin_dy, np.float32),
            "pin_cap": _np(netlist.pin_cap, np.float32), "cell_rdrv": _np(netlist.cell_rdrv, np.float32),
            "cell_fixed": _np(netlist.cell_fixed, np.uint8),
        }
        desc = _abi.NetlistDesc(self.n_cells, self.n_pins, self.n_nets,
                                *[keep[k].ctypes.data for k in ("pin_cell", "net_ptr", "pin_dir",
                                                                 "cell_type", "pin_dx", "pin_dy",
                                                                 "pin_cap", "cell_rdrv", "cell_fixed")],
                                float(netlist.r_per_um), float(netlist.c_per_um), float(netlist.d0_ps))
        handle = C.c_void_p()
        prec = _abi.TDP_FP32 if self.dtype == torch.float32 else _abi.TDP_FP64
        with torch.cuda.device(self.device):
            _abi.check("sta_build", self.lib.sta_build(C.byref(desc), prec,
                                                       C.c_void_p(self.stream.cuda_stream),
                                                       C.byref(handle)))
        self.handle = handle
        self._loss_buf = torch.zeros((), dtype=torch.float64, device=self.device)

    # ---------------------------------------------------------------- STA --
    def _pos(self, t: torch.Tensor) -> torch.Tensor:
        if t.device != self.device or t.dtype != self.dtype or not t.is_contiguous() or t.numel() != self.n_cells:
            raise ValueError(f"positions must be contiguous {self.dtype} [{self.n_cells}] on {self.device}")
        return t

    def sta_propagate(self, x: torch.Tensor, y: torch.Tensor, clock_period_ps: float, sync: bool = True):
        """Arrival / required / slack of every pin; returns (WNS, TNS) when ``sync``."""
        x, y = self._pos(x), self._pos(y)
        if sync:
            wns, tns = C.c_double(), C.c_double()
            _abi.check("sta_propagate", self.lib.sta_propagate(self.handle, _ptr(x), _ptr(y),
                                                               float(clock_period_ps), C.byref(wns),
                                                               C.byref(tns)))
            return wns.value, tns.value
        _abi.check("sta_propagate", self.lib.sta_propagate(self.handle, _ptr(x), _ptr(y),
                                                           float(clock_period_ps), None, None))
        return None

    def sta_propagate_incremental(self, x: torch.Tensor, y: torch.Tensor, clock_period_ps: float,
                                  sync: bool = True):
        """The results of sta_propagate, re-timing only what the cells that moved
        since the last propagation reach; returns (WNS, TNS) when ``sync``."""
        x, y = self._pos(x), self._pos(y)
        name = "sta_propagate_incremental"
        if sync:
            wns, tns = C.c_double(), C.c_double()
            _abi.check(name, self.lib.sta_propagate_incremental(self.handle, _ptr(x), _ptr(y),
                                                                float(clock_period_ps), C.byref(wns),
                                                                C.byref(tns)))
            return wns.value, tns.value
        _abi.check(name, self.lib.sta_propagate_incremental(self.handle, _ptr(x), _ptr(y),
                                                            float(clock_period_ps), None, None))
        return None

    def incremental_stats(self) -> dict:
        """What the last propagation re-timed (synchronises)."""
        out = (C.c_int64 * 7)()
        _abi.check("sta_incremental_stats", self.lib.sta_incremental_stats(self.handle, out))
        keys = ("full", "moved_cells", "cells_evaluated", "cells_changed", "first_level", "last_level",
                "every_cell_from_level")
        return dict(zip(keys, (int(v) for v in out)))

    def sta_get_timing(self):
        """(arr, req, slack) per pin, as new device tensors."""
        out = [torch.empty(self.n_pins, dtype=self.dtype, device=self.device) for _ in range(3)]
        _abi.check("sta_get_timing", self.lib.sta_get_timing(self.handle, *[_ptr(t) for t in out]))
        return tuple(out)

    def sta_get_net_delays(self):
        """(tnet per pin, C_load per net, driving-cell delay per net)."""
        tnet = torch.empty(self.n_pins, dtype=self.dtype, device=self.device)
        cload = torch.empty(self.n_nets, dtype=self.dtype, device=self.device)
        dnet = torch.empty(self.n_nets, dtype=self.dtype, device=self.device)
        _abi.check("sta_get_net_delays",
                   self.lib.sta_get_net_delays(self.handle, _ptr(tnet), _ptr(cload), _ptr(dnet)))
        return tnet, cload, dnet

    # --------------------------------------------------------- extraction --
    def extract_critical_paths(self, n_endpoints: int = -1, K: int = 1, keep_nonneg: bool = False,
                               sync: bool = True):
        """report_timing_endpoint(n, K); returns the number of paths when ``sync``."""
        if sync:
            n = C.c_int64()
            _abi.check("extract_critical_paths",
                       self.lib.extract_critical_paths(self.handle, int(n_endpoints), int(K),
                                                       int(bool(keep_nonneg)), C.byref(n)))
            return n.value
        _abi.check("extract_critical_paths",
                   self.lib.extract_critical_paths(self.handle, int(n_endpoints), int(K),
                                                   int(bool(keep_nonneg)), None))
        return None

    def sta_join(self):
        """The graph's stream waits for the last backward sweep (run on the
        library's second stream)."""
        _abi.check("sta_join", self.lib.sta_join(self.handle))

    def report_timing(self, n: int, keep_nonneg: bool = False) -> int:
        """report_timing(n): the n lowest-slack paths of the design, worst first;
        returns their number (the call synchronises)."""
        npth = C.c_int64()
        _abi.check("report_timing", self.lib.report_timing(self.handle, int(n), int(bool(keep_nonneg)),
                                                           C.byref(npth)))
        return npth.value

    def sta_get_paths_size(self):
        nv, npth, npin = C.c_int32(), C.c_int64(), C.c_int64()
        _abi.check("sta_get_paths_size", self.lib.sta_get_paths_size(self.handle, C.byref(nv),
                                                                     C.byref(npth), C.byref(npin)))
        return nv.value, npth.value, npin.value

    def sta_get_paths(self) -> dict:
        """Failing endpoints (sorted) and every path: ep, slack, pin_ptr, pins (start first)."""
        nv, npth, npin = self.sta_get_paths_size()
        dev = self.device
        out = {
            "viol": torch.empty(nv, dtype=torch.int32, device=dev),
            "ep": torch.empty(npth, dtype=torch.int32, device=dev),
            "slack": torch.empty(npth, dtype=self.dtype, device=dev),
            "pin_ptr": torch.empty(npth + 1, dtype=torch.int64, device=dev),
            "pins": torch.empty(max(npin, 1), dtype=torch.int32, device=dev),
        }
        _abi.check("sta_get_paths", self.lib.sta_get_paths(self.handle, _ptr(out["viol"]), _ptr(out["ep"]),
                                                           _ptr(out["slack"]), _ptr(out["pin_ptr"]),
                                                           _ptr(out["pins"])))
        out["pins"] = out["pins"][:npin]
        return out

    # ---------------------------------------------------------- pin pairs --
    def attraction_update_pairs(self, w0: float = 10.0, w1: float = 0.2, sync: bool = True):
        if sync:
            n = C.c_int64()
            _abi.check("attraction_update_pairs",
                       self.lib.attraction_update_pairs(self.handle, float(w0), float(w1), C.byref(n)))
            return n.value
        _abi.check("attraction_update_pairs",
                   self.lib.attraction_update_pairs(self.handle, float(w0), float(w1), None))
        return None

    LOSS_KINDS = {"quadratic": 0, "hpwl": 1, "euclid": 2}

    def attraction_set_loss_kind(self, kind: str):
        """Pair term of the attraction loss: "quadratic" (Eq. (9), default),
        "hpwl" or "euclid" (the ablation's alternatives)."""
        if kind not in self.LOSS_KINDS:
            raise ValueError(f"unknown loss kind {kind!r}")
        _abi.check("attraction_set_loss_kind", self.lib.attraction_set_loss_kind(self.handle, self.LOSS_KINDS[kind]))

    def attraction_reset_pairs(self):
        _abi.check("attraction_reset_pairs", self.lib.attraction_reset_pairs(self.handle))

    def attraction_set_pairs(self, pins, w):
        pins = _np(pins, np.int32)
        w = _np(w, np.float64)
        _abi.check("attraction_set_pairs",
                   self.lib.attraction_set_pairs(self.handle, len(pins), pins.ctypes.data_as(C.c_void_p),
                                                 w.ctypes.data_as(C.c_void_p)))

    def attraction_get_pairs(self):
        n = C.c_int64()
        _abi.check("attraction_get_pairs", self.lib.attraction_get_pairs(self.handle, None, None, C.byref(n)))
        pins = torch.empty(max(n.value, 1), dtype=torch.int32, device=self.device)
        w = torch.empty(max(n.value, 1), dtype=self.dtype, device=self.device)
        _abi.check("attraction_get_pairs",
                   self.lib.attraction_get_pairs(self.handle, _ptr(pins), _ptr(w), C.byref(n)))
        return pins[:n.value], w[:n.value]

    # --------------------------------------------------------------- loss --
    def attraction_loss_fwd(self, x: torch.Tensor, y: torch.Tensor, beta: float,
                            out: torch.Tensor | None = None) -> torch.Tensor:
        x, y = self._pos(x), self._pos(y)
        out = torch.empty((), dtype=torch.float64, device=self.device) if out is None else out
        _abi.check("attraction_loss_fwd",
                   self.lib.attraction_loss_fwd(self.handle, _ptr(x), _ptr(y), float(beta), _ptr(out)))
        return out

    def attraction_loss_bwd(self, x: torch.Tensor, y: torch.Tensor, beta: float,
                            grad_scale: torch.Tensor | None = None, gx=None, gy=None):
        x, y = self._pos(x), self._pos(y)
        gx = torch.empty_like(x) if gx is None else gx
        gy = torch.empty_like(y) if gy is None else gy
        if grad_scale is not None:
            grad_scale = grad_scale.detach().to(device=self.device, dtype=torch.float64).contiguous()
        _abi.check("attraction_loss_bwd",
                   self.lib.attraction_loss_bwd(self.handle, _ptr(x), _ptr(y), float(beta),
                                                _ptr(grad_scale), _ptr(gx), _ptr(gy)))
        return gx, gy

    # ------------------------------------------------------ net weighting --
    def net_weights_update(self, alpha: float = 0.5, gamma: float = 4.0, sync: bool = True):
        """One momentum update of the per-net weights from the last propagation's
        pin slacks (the net-weighting baseline); returns the number of nets
        with negative slack when ``sync``."""
        if sync:
            n = C.c_int64()
            _abi.check("net_weights_update",
                       self.lib.net_weights_update(self.handle, float(alpha), float(gamma), C.byref(n)))
            return n.value
        _abi.check("net_weights_update", self.lib.net_weights_update(self.handle, float(alpha), float(gamma), None))
        return None

    def net_weights_get(self) -> torch.Tensor:
        w = torch.empty(self.n_nets, dtype=self.dtype, device=self.device)
        _abi.check("net_weights_get", self.lib.net_weights_get(self.handle, _ptr(w)))
        return w

    def net_weights_reset(self):
        _abi.check("net_weights_reset", self.lib.net_weights_reset(self.handle))

    def attraction_loss_fwd_bwd(self, x: torch.Tensor, y: torch.Tensor, beta: float,
                                grad_scale: torch.Tensor | None = None, out=None, gx=None, gy=None):
        """attraction_loss_fwd and attraction_loss_bwd in one call (two launches);
        returns (loss device scalar, gx, gy)."""
        x, y = self._pos(x), self._pos(y)
        out = torch.empty((), dtype=torch.float64, device=self.device) if out is None else out
        gx = torch.empty_like(x) if gx is None else gx
        gy = torch.empty_like(y) if gy is None else gy
        if grad_scale is not None:
            grad_scale = grad_scale.detach().to(device=self.device, dtype=torch.float64).contiguous()
        _abi.check("attraction_loss_fwd_bwd",
                   self.lib.attraction_loss_fwd_bwd(self.handle, _ptr(x), _ptr(y), float(beta), _ptr(grad_scale),
                                                    _ptr(out), _ptr(gx), _ptr(gy)))
        return out, gx, gy

    # ---------------------------------------------------- instrumentation --
    def tdp_get_launch_count(self) -> int:
        n = C.c_int64()
        _abi.check("tdp_get_launch_count", self.lib.tdp_get_launch_count(self.handle, C.byref(n)))
        return n.value

    def tdp_profile_kernel(self, name: str | None):
        _abi.check("tdp_profile_kernel",
                   self.lib.tdp_profile_kernel(self.handle, None if not name else name.encode()))

    def tdp_profile_read(self):
        """(number of timed launches, their summed device time in ms); resets."""
        n, ms = C.c_int64(), C.c_double()
        _abi.check("tdp_profile_read", self.lib.tdp_profile_read(self.handle, C.byref(n), C.byref(ms)))
        return n.value, ms.value

    # ----------------------------------------------------------- lifetime --
    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.sta_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class AttractionLoss(torch.autograd.Function):
    """PP(x, y) = beta * sum w Q over the pin-pair set P (Eq. (9)).

    forward calls ``attraction_loss_fwd``; backward calls the hand-written
    adjoint ``attraction_loss_bwd`` with the incoming gradient as a device
    scalar (no host synchronisation).  P and w are constants of the step.
    """

    @staticmethod
    def forward(ctx, x, y, graph: TimingGraph, beta: float):
        ctx.graph, ctx.beta = graph, beta
        ctx.save_for_backward(x, y)
        return graph.attraction_loss_fwd(x.detach(), y.detach(), beta)

    @staticmethod
    def backward(ctx, g):
        x, y = ctx.saved_tensors
        gx, gy = ctx.graph.attraction_loss_bwd(x.detach(), y.detach(), ctx.beta, grad_scale=g)
        return gx, gy, None, None


def attraction_loss(graph: TimingGraph, x: torch.Tensor, y: torch.Tensor, beta: float = 2.5e-5):
    return AttractionLoss.apply(x, y, graph, beta)
