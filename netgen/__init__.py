"""Seeded synthetic netlist generator shared by the oracle and the CUDA path.

This module draws random netlist topology and random per-cell / per-pin values
only.  It contains none of the timing, path or loss arithmetic of the method:
no delay, arrival, slack, path or weight is computed here.  Both the FP64 CPU
oracle (``oracle/``) and the CUDA library consume its output unchanged.

The netlists stand in for the ICCAD 2015 ``superblue`` designs of Section IV
(not available here).  Shape of every netlist (one recipe, five sizes):

* movable cells = combinational cells (1, 2, 3 or 4 inputs, uniform) plus
  flip-flops (one D input, one Q output);
* ``n_nets - n_cells`` extra nets are driven by fixed primary-input ports (PI);
* combinational cells are spread evenly over logic levels 1..D; input 0 of a
  level-l cell is driven from level l-1 (so every cell sits exactly on level l
  and a chain of depth D exists); the other inputs pick level l-1 with
  probability 0.5, level 0 (flip-flop Q / PI) with probability 0.2, else a
  uniform level in [0, l-1];
* flip-flop D pins pick a driver level uniformly in [1, D];
* within a driver level every net first receives one sink (coverage); the
  remaining slots go to high-fanout nets up to their drawn fanout, then to the
  other nets with probability proportional to (drawn fanout - 1);
* a net left without any sink gets a fixed primary-output port (PO) as its sink;
* drawn fanout: geometric(p) capped, and a fraction of nets with a truncated
  Pareto(alpha=2) fanout on [64, 1000];
* cell positions uniform on a 1000 x 1000 um die; R_drv ~ U[0.5, 2] kOhm;
  pin capacitance ~ U[1, 3] fF; optional pin offsets ~ U[-1, 1] um;
  wire r = 0.004 kOhm/um, c = 0.2 fF/um, d0 = 5 ps.

Pins are numbered net-contiguously: net ``e`` owns pins
``net_ptr[e] .. net_ptr[e+1]-1`` and its first pin is the driver.
"""
from __future__ import annotations

from dataclasses import dataclass, field, asdict
import numpy as np

COMB, FF, PI, PO = 0, 1, 2, 3
SINK, DRIVER = 0, 1

DIE_UM = 1000.0


@dataclass(frozen=True)
class NetlistConfig:
    name: str
    n_cells: int          # movable cells: combinational + flip-flops
    n_ff: int
    n_nets: int
    depth: int
    p_geom: float         # geometric fanout parameter
    fanout_cap: int       # cap of the geometric fanout
    hf_frac: float        # fraction of nets with a Pareto fanout on [64, 1000]
    t_factor: float       # clock period = t_factor x max endpoint arrival
    K: int                # paths per violating endpoint
    offsets: bool = True  # random pin offsets (else all zero)
    r_per_um: float = 0.004
    c_per_um: float = 0.2
    d0_ps: float = 5.0


CONFIGS = {
    # 2,000 cells (200 FF), 2,200 nets, ~7k pins, depth 30, fanout geometric p=0.5 on 1..8
    "tiny": NetlistConfig("tiny", 2_000, 200, 2_200, 30, 0.5, 8, 0.0, 0.9, 4, offsets=False),
    # 20,000 cells, 22,000 nets, ~75k pins, depth 40
    "diff": NetlistConfig("diff", 20_000, 2_000, 22_000, 40, 0.5, 8, 0.0, 0.9, 8),
    # 200,000 cells (10% FF), 220,000 nets, ~750k pins, depth 60, geometric p=0.4 capped at 32
    "mid": NetlistConfig("mid", 200_000, 20_000, 220_000, 60, 0.4, 32, 0.0, 0.85, 16),
    # 1.2M cells (8% FF), 1.3M nets, ~4.5M pins, depth 80, 0.5% nets of fanout 64-1000
    "1.2M": NetlistConfig("1.2M", 1_200_000, 96_000, 1_300_000, 80, 0.4, 32, 0.005, 0.85, 16),
    # 3M cells (8% FF), 3.3M nets, ~11M pins, depth 120, clock at 0.8x max arrival, K=32
    "stress": NetlistConfig("stress", 3_000_000, 240_000, 3_300_000, 120, 0.4, 32, 0.005, 0.8, 32),
}


@dataclass
class Netlist:
    """Host arrays in the layout the C-ABI ``tdp_netlist_desc`` expects."""
    n_cells: int
    n_pins: int
    n_nets: int
    pin_cell: np.ndarray   # int32[n_pins]
    net_ptr: np.ndarray    # int32[n_nets+1]
    pin_dir: np.ndarray    # uint8[n_pins]   1 = driver (first pin of its net)
    cell_type: np.ndarray  # int32[n_cells]  COMB / FF / PI / PO
    pin_dx: np.ndarray     # float32[n_pins] um
    pin_dy: np.ndarray     # float32[n_pins] um
    pin_cap: np.ndarray    # float32[n_pins] fF
    cell_rdrv: np.ndarray  # float32[n_cells] kOhm
    cell_fixed: np.ndarray # uint8[n_cells]
    x: np.ndarray          # float32[n_cells] initial placement, um
    y: np.ndarray          # float32[n_cells]
    r_per_um: float
    c_per_um: float
    d0_ps: float
    meta: dict = field(default_factory=dict)

    def stats(self) -> dict:
        fan = np.diff(self.net_ptr) - 1
        ct = self.cell_type
        return {
            "cells": int(self.n_cells), "pins": int(self.n_pins), "nets": int(self.n_nets),
            "comb": int((ct == COMB).sum()), "ff": int((ct == FF).sum()),
            "pi": int((ct == PI).sum()), "po": int((ct == PO).sum()),
            "max_fanout": int(fan.max()), "mean_fanout": float(fan.mean()),
            "nets_fanout_ge64": int((fan >= 64).sum()),
        }


def _truncated_pareto(rng, n, lo=64.0, hi=1000.0, alpha=2.0):
    u = rng.random(n)
    # inverse CDF of Pareto(alpha, lo) truncated at hi
    tail = 1.0 - (lo / hi) ** alpha
    return np.floor(lo / (1.0 - u * tail) ** (1.0 / alpha)).astype(np.int64)


def generate(cfg: NetlistConfig | str, seed: int = 1) -> Netlist:
    """Draw one netlist of the given configuration (deterministic in ``seed``)."""
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    rng = np.random.default_rng(seed)
    D = cfg.depth
    n_comb = cfg.n_cells - cfg.n_ff
    n_pi = cfg.n_nets - cfg.n_cells
    assert n_comb >= D and n_pi >= 0

    # ---- driver entities: comb cells, flip-flops, primary inputs (one net each)
    sizes = np.full(D, n_comb // D, dtype=np.int64)
    sizes[: n_comb % D] += 1
    comb_level = np.repeat(np.arange(1, D + 1, dtype=np.int64), sizes)
    n_drv = n_comb + cfg.n_ff + n_pi
    drv_level = np.concatenate([comb_level, np.zeros(cfg.n_ff + n_pi, dtype=np.int64)])

    # drawn fanout of every driver's net
    fan = rng.geometric(cfg.p_geom, size=n_drv)
    fan = np.minimum(fan, cfg.fanout_cap).astype(np.int64)
    hf = rng.random(n_drv) < cfg.hf_frac
    fan[hf] = _truncated_pareto(rng, int(hf.sum()))

    # ---- sink slots: comb inputs, then flip-flop D pins
    fanin = rng.integers(1, 5, size=n_comb)
    slot_cell = np.repeat(np.arange(n_comb, dtype=np.int64), fanin)     # consumer comb index
    first = np.concatenate([[0], np.cumsum(fanin)[:-1]])
    slot_k = np.arange(slot_cell.size) - np.repeat(first, fanin)
    lvl = comb_level[slot_cell]
    u = rng.random(slot_cell.size)
    any_lower = np.floor(rng.random(slot_cell.size) * lvl).astype(np.int64)  # uniform in [0, l-1]
    choose = np.where(u < 0.5, lvl - 1, np.where(u < 0.7, 0, any_lower))
    choose[slot_k == 0] = lvl[slot_k == 0] - 1
    n_comb_slots = slot_cell.size
    ff_choose = rng.integers(1, D + 1, size=cfg.n_ff)
    slot_level = np.concatenate([choose, ff_choose])
    n_slots = slot_level.size
    slot_drv = np.full(n_slots, -1, dtype=np.int64)

    order = np.argsort(slot_level, kind="stable")
    bounds = np.searchsorted(slot_level[order], np.arange(D + 2))
    drv_order = np.argsort(drv_level, kind="stable")
    dbounds = np.searchsorted(drv_level[drv_order], np.arange(D + 2))
    for L in range(D + 1):
        slots = order[bounds[L]: bounds[L + 1]]
        slots = slots[rng.permutation(slots.size)]
        nets = drv_order[dbounds[L]: dbounds[L + 1]]
        if slots.size == 0 or nets.size == 0:
            continue
        c = min(slots.size, nets.size)
        slot_drv[slots[:c]] = rng.permutation(nets)[:c]           # coverage
        rest = slots[c:]
        if rest.size == 0:
            continue
        hf_nets = nets[hf[nets]]
        stubs = np.repeat(hf_nets, np.maximum(fan[hf_nets] - 1, 0))
        stubs = stubs[rng.permutation(stubs.size)]
        h = min(rest.size, stubs.size)
        slot_drv[rest[:h]] = stubs[:h]
        rest = rest[h:]
        if rest.size == 0:
            continue
        norm = nets[~hf[nets]]
        if norm.size == 0:
            norm = nets
        wgt = (fan[norm] - 1).astype(np.float64)
        if wgt.sum() <= 0:
            wgt = np.ones(norm.size)
        slot_drv[rest] = rng.choice(norm, size=rest.size, p=wgt / wgt.sum())
    assert (slot_drv >= 0).all()

    # ---- primary outputs for nets left without a sink
    cnt = np.bincount(slot_drv, minlength=n_drv)
    po_drv = np.nonzero(cnt == 0)[0]
    n_po = po_drv.size

    # ---- cell ids: comb | ff | pi | po, then a random relabelling
    n_all = cfg.n_cells + n_pi + n_po
    ctype_pre = np.concatenate([np.full(n_comb, COMB), np.full(cfg.n_ff, FF),
                                np.full(n_pi, PI), np.full(n_po, PO)]).astype(np.int32)
    cell_perm = rng.permutation(n_all)            # pre-index -> cell id
    cell_type = np.empty(n_all, dtype=np.int32)
    cell_type[cell_perm] = ctype_pre
    drv_cell = cell_perm[np.arange(n_drv)]         # driver entity -> cell id
    # sink slots -> consumer cell id
    slot_cons = np.concatenate([cell_perm[slot_cell], cell_perm[n_comb + np.arange(cfg.n_ff)]])
    po_cells = cell_perm[cfg.n_cells + n_pi + np.arange(n_po)]

    # ---- net ids: random relabelling of driver entities
    net_of_drv = rng.permutation(n_drv)
    sink_net = np.concatenate([net_of_drv[slot_drv], net_of_drv[po_drv]])
    sink_cell = np.concatenate([slot_cons, po_cells])
    # within a consumer cell keep input order by slot order; random order of sinks inside a net
    tie = rng.random(sink_net.size)
    sorder = np.lexsort((tie, sink_net))
    sink_net = sink_net[sorder]
    sink_cell = sink_cell[sorder]
    fanout = np.bincount(sink_net, minlength=n_drv)
    net_ptr = np.zeros(n_drv + 1, dtype=np.int64)
    net_ptr[1:] = np.cumsum(fanout + 1)
    n_pins = int(net_ptr[-1])
    pin_cell = np.empty(n_pins, dtype=np.int32)
    pin_dir = np.zeros(n_pins, dtype=np.uint8)
    drv_of_net = np.empty(n_drv, dtype=np.int64)
    drv_of_net[net_of_drv] = np.arange(n_drv)
    pin_cell[net_ptr[:-1]] = drv_cell[drv_of_net]
    pin_dir[net_ptr[:-1]] = DRIVER
    sink_pos = np.repeat(net_ptr[:-1] + 1, fanout) + (np.arange(sink_net.size) -
                                                       np.repeat(np.concatenate([[0], np.cumsum(fanout)[:-1]]), fanout))
    pin_cell[sink_pos] = sink_cell

    # ---- per-cell and per-pin values
    rdrv = rng.uniform(0.5, 2.0, size=n_all).astype(np.float32)
    rdrv[cell_type == PO] = 0.0
    cap = rng.uniform(1.0, 3.0, size=n_pins).astype(np.float32)
    if cfg.offsets:
        dx = rng.uniform(-1.0, 1.0, size=n_pins).astype(np.float32)
        dy = rng.uniform(-1.0, 1.0, size=n_pins).astype(np.float32)
    else:
        dx = np.zeros(n_pins, dtype=np.float32)
        dy = np.zeros(n_pins, dtype=np.float32)
    fixed = ((cell_type == PI) | (cell_type == PO)).astype(np.uint8)
    x = rng.uniform(0.0, DIE_UM, size=n_all).astype(np.float32)
    y = rng.uniform(0.0, DIE_UM, size=n_all).astype(np.float32)

    return Netlist(
        n_cells=n_all, n_pins=n_pins, n_nets=n_drv,
        pin_cell=pin_cell, net_ptr=net_ptr.astype(np.int32), pin_dir=pin_dir,
        cell_type=cell_type, pin_dx=dx, pin_dy=dy, pin_cap=cap, cell_rdrv=rdrv,
        cell_fixed=fixed, x=x, y=y,
        r_per_um=cfg.r_per_um, c_per_um=cfg.c_per_um, d0_ps=cfg.d0_ps,
        meta={"config": asdict(cfg), "seed": seed},
    )


def perturb(x: np.ndarray, y: np.ndarray, fixed: np.ndarray, sigma: float, rng) -> tuple:
    """One seeded Gaussian move of every movable cell, clamped to the die."""
    mv = fixed == 0
    nx = x.copy()
    ny = y.copy()
    nx[mv] = np.clip(x[mv] + rng.normal(0.0, sigma, size=int(mv.sum())), 0.0, DIE_UM)
    ny[mv] = np.clip(y[mv] + rng.normal(0.0, sigma, size=int(mv.sum())), 0.0, DIE_UM)
    return nx.astype(x.dtype), ny.astype(y.dtype)


def from_lists(cells: list, nets: list, r_per_um=0.004, c_per_um=0.2, d0_ps=5.0) -> Netlist:
    """Build a hand-written netlist.

    ``cells``: list of dicts ``{"type": "COMB"|"FF"|"PI"|"PO", "x", "y", "rdrv"}``.
    ``nets``: list of lists of pins; each pin is ``(cell_index, cap_fF[, dx, dy])``;
    the first pin of a net is its driver.
    """
    tmap = {"COMB": COMB, "FF": FF, "PI": PI, "PO": PO}
    pin_cell, pin_dir, cap, dx, dy, net_ptr = [], [], [], [], [], [0]
    for net in nets:
        for k, p in enumerate(net):
            pin_cell.append(p[0])
            pin_dir.append(DRIVER if k == 0 else SINK)
            cap.append(p[1])
            dx.append(p[2] if len(p) > 2 else 0.0)
            dy.append(p[3] if len(p) > 3 else 0.0)
        net_ptr.append(len(pin_cell))
    ct = np.array([tmap[c["type"]] for c in cells], dtype=np.int32)
    return Netlist(
        n_cells=len(cells), n_pins=len(pin_cell), n_nets=len(nets),
        pin_cell=np.array(pin_cell, dtype=np.int32), net_ptr=np.array(net_ptr, dtype=np.int32),
        pin_dir=np.array(pin_dir, dtype=np.uint8), cell_type=ct,
        pin_dx=np.array(dx, dtype=np.float32), pin_dy=np.array(dy, dtype=np.float32),
        pin_cap=np.array(cap, dtype=np.float32),
        cell_rdrv=np.array([c.get("rdrv", 0.0) for c in cells], dtype=np.float32),
        cell_fixed=((ct == PI) | (ct == PO)).astype(np.uint8),
        x=np.array([c["x"] for c in cells], dtype=np.float32),
        y=np.array([c["y"] for c in cells], dtype=np.float32),
        r_per_um=r_per_um, c_per_um=c_per_um, d0_ps=d0_ps,
    )


def random_dag(n_comb: int, n_ff: int, depth: int, wide_frac: float, seed: int = 1,
               max_inputs: int = 10) -> Netlist:
    """A small seeded levelized netlist whose combinational cells include
    wide ones: a fraction ``wide_frac`` of them has 5 to ``max_inputs``
    inputs, the rest 1 to 4.  Input 0 of a level-l cell comes from level
    l - 1 (flip-flop Q for level 1), the others from a uniform lower level;
    every flip-flop D pin from a uniform combinational cell; a net left
    without a sink gets a primary-output port.  Positions uniform on the die,
    R_drv ~ U[0.5, 2] kOhm, pin capacitance ~ U[1, 3] fF, zero pin offsets."""
    rng = np.random.default_rng(seed)
    cells = [{"type": "FF", "x": rng.uniform(0, DIE_UM), "y": rng.uniform(0, DIE_UM),
              "rdrv": rng.uniform(0.5, 2.0)} for _ in range(n_ff)]
    by_level = [list(range(n_ff))]
    inputs = {}
    for l in range(1, depth + 1):
        n_l = n_comb // depth + (1 if l <= n_comb % depth else 0)
        lvl = []
        for _ in range(n_l):
            c = len(cells)
            cells.append({"type": "COMB", "x": rng.uniform(0, DIE_UM), "y": rng.uniform(0, DIE_UM),
                          "rdrv": rng.uniform(0.5, 2.0)})
            k = int(rng.integers(5, max_inputs + 1)) if rng.random() < wide_frac else int(rng.integers(1, 5))
            drv = [by_level[l - 1][int(rng.integers(len(by_level[l - 1])))]]
            for _ in range(k - 1):
                ll = int(rng.integers(0, l))
                drv.append(by_level[ll][int(rng.integers(len(by_level[ll])))])
            inputs[c] = drv
            lvl.append(c)
        by_level.append(lvl)
    comb = [c for lvl in by_level[1:] for c in lvl]
    for f in range(n_ff):
        inputs[f] = [comb[int(rng.integers(len(comb)))]]
    sinks = {c: [] for c in range(len(cells))}
    for c, drv in inputs.items():
        for d in drv:
            sinks[d].append(c)
    n_driving = len(cells)
    for d in range(n_driving):
        if not sinks[d]:
            cells.append({"type": "PO", "x": rng.uniform(0, DIE_UM), "y": rng.uniform(0, DIE_UM), "rdrv": 0.0})
            sinks[d].append(len(cells) - 1)
    nets = []
    for d in range(n_driving):
        order = rng.permutation(len(sinks[d]))
        nets.append([(d, float(rng.uniform(1.0, 3.0)))] +
                    [(sinks[d][i], float(rng.uniform(1.0, 3.0))) for i in order])
    return from_lists(cells, nets)
