#!/usr/bin/env python
"""Timing iterations per second of the timing-driven placement hot path.

One step = one timing iteration of the method on one synthetic netlist:
    sta_propagate -> extract_critical_paths (report_timing_endpoint(all, K))
    -> attraction_update_pairs (Eq. w_ij) -> attraction_loss_fwd_bwd (Eq. 9, loss and gradient)
at a new placement every step (seeded Gaussian moves, sigma = 2 um).  The
workload is the 1.2M-cell netlist (1.3M nets, ~4.2M pins, depth 80, 0.5% nets
of fanout 64-1000, clock at 0.85x the largest arrival, K = 16).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs as independent replicas (one netlist per rank, no collective in
the data path); launch with torch.distributed.run.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import signal
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "STA+path-extract+attraction fwd/bwd iters/sec at 1.2M cells; % HBM roofline"
UNIT = "iter/s"
W0, W1, BETA, SIGMA = 10.0, 0.2, 2.5e-5, 2.0
N_POS_SETS = 32            # distinct placements cycled through by the timed loop
ROOFLINE_KERNEL = "fwd_sweep"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default="1.2M")
    ap.add_argument("--K", type=int, default=None, help="paths per failing endpoint (default: the config's)")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--roofline-kernel", default=ROOFLINE_KERNEL)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--stages", action="store_true", help="also time each entry point (diagnostic)")
    ap.add_argument("--no-table1", action="store_true",
                    help="skip Table I's comparison of report_timing(n) with report_timing_endpoint(n, k)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-on-GPU comparison run")
    ap.add_argument("--no-incremental", action="store_true",
                    help="skip the incremental-timing measurements (sta_propagate_incremental)")
    return ap.parse_args()


# ---------------------------------------------------------------- helpers --

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(value: float, world: int, device) -> float:
    """Max over ranks (identity for one rank)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(ms_local: float, steps: int, world: int, device) -> tuple:
    """Slowest rank's time for `steps` steps, and whole-job iterations / s
    (every rank runs its own replica of the workload)."""
    ms = reduce_max(ms_local, world, device)
    return ms, world * steps / (ms / 1000.0)


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL,
                start_new_session=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        try:
            os.killpg(self.proc.pid, signal.SIGTERM)
        except OSError:
            pass
        self.proc.wait(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload_desc(cfg, nl):
    st = nl.stats()
    K = cfg.K
    return {"workload": f"{cfg.name}: {st['cells']:,} cells ({cfg.n_ff:,} FF, {st['pi']:,} PI, {st['po']:,} PO), "
                        f"{st['nets']:,} nets, {st['pins']:,} pins, depth {cfg.depth}, K={K}, "
                        f"clock {cfg.t_factor}x max arrival",
            "cells": st["cells"], "nets": st["nets"], "pins": st["pins"], "depth": cfg.depth, "K": K,
            "max_fanout": st["max_fanout"], "t_factor": cfg.t_factor}


# ------------------------------------------------------ algorithmic bytes --

# A level sweep is one cooperative launch over all logic levels (or, with
# TDP_LEVEL_GRAPHS=1, one CUDA-graph replay of a kernel per level); its
# "launch" for the roofline is the whole sweep.
LAUNCH_UNIT = {"fwd_sweep": "one forward sweep over all logic levels (a single cooperative launch)",
               "bwd_sweep": "one backward sweep over all logic levels (a single cooperative launch)"}

# DRAM bytes (read + write) per launch from ncu captures, by (workload, K),
# with the SHA-256 of the sources the kernel was built from when it was
# taken; a figure is reported only for its workload and while those sources
# are unchanged.
SWEEP_SOURCES = ["paper_2503_11674_b300/csrc/tdp_sta.cu", "paper_2503_11674_b300/csrc/tdp_internal.cuh"]
PAIR_SOURCES = ["paper_2503_11674_b300/csrc/tdp_pairs.cu", "paper_2503_11674_b300/csrc/tdp_internal.cuh"]
PROFILED_TRAFFIC = {
    ("1.2M", 16): {
        "fwd_sweep": {"bytes": 511739904, "sources": SWEEP_SOURCES, "sha256": "b8921e57515016b5f8badf95eb604b68446769a956cc9ad52825b0a4428d7111"},
        "bwd_sweep": {"bytes": 128792320, "sources": SWEEP_SOURCES, "sha256": "b8921e57515016b5f8badf95eb604b68446769a956cc9ad52825b0a4428d7111"},
        "pair_walk": {"bytes": 22054656, "sources": PAIR_SOURCES, "sha256": "79052c62d3f43c9ac0b1a3deaf7fe13d9affae0679230929a60ea0962ff4a9b3"},
    },
    ("stress", 32): {
        "fwd_sweep": {"bytes": 2477957704, "sources": SWEEP_SOURCES, "sha256": "b8921e57515016b5f8badf95eb604b68446769a956cc9ad52825b0a4428d7111"},
    },
}


def profiled_traffic(kernel: str, workload=("1.2M", 16)):
    import hashlib
    rec = PROFILED_TRAFFIC.get(tuple(workload), {}).get(kernel)
    if rec is None:
        return None
    h = hashlib.sha256()
    for src in rec["sources"]:
        with open(os.path.join(ROOT, src), "rb") as f:
            h.update(f.read())
    if h.hexdigest() != rec["sha256"]:
        return None
    return rec["bytes"]


def list_length(K: int) -> int:
    """Sidetrack entries kept per node for top-K (the library's length buckets)."""
    return next(b for b in (0, 3, 7, 15, 31) if b >= K - 1)


def netlist_counts(nl) -> dict:
    """Element counts the byte models are stated in."""
    import numpy as np
    C, P, N = nl.n_cells, nl.n_pins, nl.n_nets
    S = P - N
    sink_cell_type = nl.cell_type[nl.pin_cell[nl.pin_dir == 0]]
    n_in = int((sink_cell_type == 0).sum())          # inputs of combinational cells
    return {"cells": C, "pins": P, "nets": N, "sinks": S, "comb_inputs": n_in, "endpoints": int(S - n_in),
            "comb": int((nl.cell_type == 0).sum())}


# The method's own traffic model: the compulsory bytes of each step of the
# timing iteration, each array element touched once, FP32 values and 4-byte
# indices, per element (the step names follow the hot-path table):
#   a1+a2 net RC       read 28 B per sink and 28 B per net, write 4 B per sink and 4 B per net
#   a3+a4 forward      read 16 B per cell input pin and 8 B per cell, write 4 B per pin and 8 B per cell
#   a5 backward        12 B per pin
#   a6 slack, WNS/TNS  12 B per pin (here: per endpoint; other pins' slacks are formed on request)
#   a7-a10 extraction and pair update
#                      20 B per pair occurrence (a net arc on an extracted path) for the
#                      search and 32 B per occurrence for the pair update (4 radix passes x 8 B)
#   a11 loss           40 B per pair; the backward pass also 8 B per pin and 8 B per cell
# The sidetrack lists of the forward sweep are not part of a3+a4: they are
# the top-K search's data (a9), moved into the sweep by this design, and are
# reported on their own.
MODEL_STEPS = {
    "net_rc": "a1+a2", "fwd_sweep": "a3+a4", "bwd_sweep": "a5", "ep_wns": "a6 (endpoints)",
    "topk+pair_walk": "a7-a10", "pp_fwd_bwd": "a11 forward + backward",
}


def model_bytes(step: str, nl, g_info: dict) -> float:
    """Bytes of one launch of `step` by the method's traffic model above."""
    c = netlist_counts(nl)
    if step == "net_rc":
        return 32 * c["sinks"] + 32 * c["nets"]
    if step == "fwd_sweep":
        return 16 * c["comb_inputs"] + 8 * c["comb"] + 4 * c["pins"] + 8 * c["comb"]
    if step == "bwd_sweep":
        return 12 * c["pins"]
    if step == "ep_wns":
        return 12 * c["endpoints"]
    if step == "topk+pair_walk":
        return (20 + 32) * g_info["path_pins"] / 2.0
    if step == "pp_fwd_bwd":
        return 40 * g_info["pairs"] + 40 * g_info["pairs"] + 8 * c["pins"] + 8 * c["cells"]
    raise ValueError(step)


def list_bytes(nl, g_info: dict) -> float:
    """Sidetrack-list bytes of one forward sweep: per combinational cell the
    inherited list read and its own list written, L entries of 8 B each."""
    return netlist_counts(nl)["comb"] * 16 * g_info["list_L"]


def own_bytes(kernel: str, nl, g_info: dict) -> float:
    """This design's compulsory DRAM bytes of one launch of `kernel` (FP32
    graph, 4-byte indices): every array element the kernel as built must read
    or write, counted once; gathers of shared data (cell positions, driver
    arrival) are counted once per element of the gathered array.  Unlike the
    method's model above this includes the design's own data (sidetrack
    lists, padded records, compacted pair lists).
    """
    import numpy as np
    C, P, N = nl.n_cells, nl.n_pins, nl.n_nets
    S = P - N
    n_start = int(np.isin(nl.cell_type[nl.pin_cell[nl.net_ptr[:-1]]], (1, 2)).sum())
    sink_cell_type = nl.cell_type[nl.pin_cell[nl.pin_dir == 0]]
    n_in = int((sink_cell_type == 0).sum())          # inputs of combinational cells
    n_ep = int(S - n_in)                              # flip-flop D and primary-output pins
    n_comb = int((nl.cell_type == 0).sum())
    if kernel == "fwd_sweep":
        # per combinational cell: input range, output pin and net (12), its
        # delay (4), arrival of the output (8), worst input / chain length (12);
        # sidetrack list: write L entries and read the inherited L (8 B each)
        # and both counts (8); per input: pin, net, driver, driver kind (13),
        # Elmore delay (4) (its arrival is formed on request, not stored);
        # per driving net: its arrival (8) and chain length (4), each read once
        L = g_info["list_L"]
        return n_comb * (12 + 4 + 8 + 12 + 16 * L + 8) + n_in * (13 + 4) + N * (8 + 4)
    if kernel == "bwd_sweep":
        # per sink: kind, cell output, its net (9), Elmore delay (4); per net:
        # its required time written (8) and the driving cell's delay (4); per
        # comb output its required time read once (8).  Only nets' required
        # times are stored: pins' required times and slacks (other than the
        # endpoints', from ep_wns) are formed on request
        return S * (9 + 4) + N * (8 + 4) + n_comb * 8
    if kernel == "ep_wns":
        # per endpoint: (pin, driver pin) (8), driver arrival (8), Elmore delay
        # (4), arrival, required time and slack written (20)
        return n_ep * 40
    if kernel == "net_rc":
        return (4 * (N + 1) + 4 * P + 8 * P + 4 * S + 8 * C + 4 * N + N
                + 4 * S + 4 * N + 4 * N + 8 * n_start)
    if kernel == "pair_walk":
        occ = g_info["path_pins"] / 2.0                 # sink pins on paths = net arcs
        paths = g_info["paths"]
        # per net arc: pred_in + pred_net of the driver (8) and two 8-byte
        # read-modify-writes (32; the raised maximum marks the sink touched);
        # per path: its endpoint, slack, cost, count and parent / sidetrack
        # records (24)
        return occ * 40.0 + paths * 24.0
    if kernel == "pp_fwd":
        # per pair: its list entry (4), its net and the net's driver (8), the
        # two pins' cells (8), offsets (16) and the weight (4), the two cells'
        # positions (16)
        nP = g_info["pairs"]
        return 56 * nP
    if kernel == "pp_bwd_net":
        # per pair as the forward pass (56) and its gradient slot (4 + 8
        # written); per pair net the driver's slot (4 + 8 written)
        nP = g_info["pairs"]
        return 68 * nP + 12 * min(nP, N)
    if kernel == "pp_fwd_bwd":
        # the loss and the per-pair gradients in one pass over the records:
        # per pair as the backward pass (68), per pair net the driver's slot
        nP = g_info["pairs"]
        return 68 * nP + 12 * min(nP, N)
    if kernel == "pp_bwd_cell":
        return 4 * (C + 1) + 8 * P + C + 8 * C
    if kernel == "topk":
        return g_info["viol"] * (4 + 4 + 4 + 4 + 1) + g_info["paths"] * (16 + 8 + 16)
    raise ValueError(kernel)


# ------------------------------------------------------------------- ours --

def run_ours(args):
    import numpy as np
    import torch

    import netgen
    from paper_2503_11674_b300 import TimingGraph

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    cfg = netgen.CONFIGS[args.config]
    if args.K:
        import dataclasses
        cfg = dataclasses.replace(cfg, K=args.K)
    seed = args.seed + rank                       # independent replica per rank
    nl = netgen.generate(cfg, seed)
    G = TimingGraph(nl, "fp32", device=dev)
    n = nl.n_cells

    # placements: a seeded random walk of the movable cells, resident on the device
    gen = torch.Generator(device=dev)
    gen.manual_seed(1000 + seed)
    mv = torch.tensor(nl.cell_fixed == 0, device=dev)
    xs = torch.empty((N_POS_SETS, n), dtype=torch.float32, device=dev)
    ys = torch.empty((N_POS_SETS, n), dtype=torch.float32, device=dev)
    x = torch.tensor(nl.x, device=dev)
    y = torch.tensor(nl.y, device=dev)
    for k in range(N_POS_SETS):
        x = torch.where(mv, (x + SIGMA * torch.randn(n, generator=gen, device=dev)).clamp(0, netgen.DIE_UM), x)
        y = torch.where(mv, (y + SIGMA * torch.randn(n, generator=gen, device=dev)).clamp(0, netgen.DIE_UM), y)
        xs[k].copy_(x)
        ys[k].copy_(y)
    # clock period from this placement: with T = 0 every endpoint fails and
    # WNS = -(largest endpoint arrival)
    wns0, _ = G.sta_propagate(xs[0], ys[0], 0.0)
    T = cfg.t_factor * (-wns0)
    K = cfg.K
    loss_buf = torch.zeros((), dtype=torch.float64, device=dev)
    gx = torch.empty(n, dtype=torch.float32, device=dev)
    gy = torch.empty(n, dtype=torch.float32, device=dev)

    def step(k):
        xk, yk = xs[k % N_POS_SETS], ys[k % N_POS_SETS]
        G.sta_propagate(xk, yk, T, sync=False)
        G.extract_critical_paths(-1, K, False, sync=False)
        G.attraction_update_pairs(W0, W1, sync=False)
        G.attraction_loss_fwd_bwd(xk, yk, BETA, out=loss_buf, gx=gx, gy=gy)

    stream = torch.cuda.current_stream(dev)
    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize(dev)

    # sizes of the per-step work (for the roofline units), from the last warm-up step
    n_viol, n_paths, n_path_pins = G.sta_get_paths_size()
    info = {"viol": n_viol, "paths": n_paths, "path_pins": n_path_pins, "list_L": list_length(K)}

    # ------------------------------------------------ device-timed region --
    G.tdp_profile_kernel(args.roofline_kernel)
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = G.tdp_get_launch_count()
    barrier(world)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        step(args.warmup + k)
    G.sta_join()  # the last step's backward sweep (on the library's second stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    ms_local = e0.elapsed_time(e1)
    launches = G.tdp_get_launch_count() - launches0
    clk = clocks.stop()
    prof_n, prof_ms = G.tdp_profile_read()
    G.tdp_profile_kernel(None)
    ms, value = aggregate(ms_local, args.steps, world, dev)
    n_pairs = G.attraction_get_pairs()[0].numel()
    info["pairs"] = n_pairs
    wns, tns = G.sta_propagate(xs[0], ys[0], T)

    # ------------------------------------- end to end through host buffers --
    # Every step copies its positions in from pinned host memory and its
    # loss and gradient out to pinned host memory.  The copies run on a
    # second stream, double-buffered: the next step's positions are copied
    # in, and this step's results copied out, while the library computes.
    xh = torch.empty((N_POS_SETS, n), dtype=torch.float32, pin_memory=True)
    yh = torch.empty((N_POS_SETS, n), dtype=torch.float32, pin_memory=True)
    xh.copy_(xs)
    yh.copy_(ys)
    copy = torch.cuda.Stream(dev)
    xd = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(2)]
    yd = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(2)]
    gxd = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(2)]
    gyd = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(2)]
    lossd = [torch.zeros((), dtype=torch.float64, device=dev) for _ in range(2)]
    gxh = [torch.empty(n, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    gyh = [torch.empty(n, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    lossh = [torch.empty((), dtype=torch.float64, pin_memory=True) for _ in range(2)]
    h2d = [torch.cuda.Event() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    d2h = [torch.cuda.Event() for _ in range(2)]
    e2e_steps = max(1, min(args.steps, 100))

    def e2e_run(n_steps):
        with torch.cuda.stream(copy):
            xd[0].copy_(xh[0], non_blocking=True)
            yd[0].copy_(yh[0], non_blocking=True)
        h2d[0].record(copy)
        for k in range(n_steps):
            b = k % 2
            stream.wait_event(h2d[b])
            G.sta_propagate(xd[b], yd[b], T, sync=False)
            G.extract_critical_paths(-1, K, False, sync=False)
            G.attraction_update_pairs(W0, W1, sync=False)
            G.attraction_loss_fwd_bwd(xd[b], yd[b], BETA, out=lossd[b], gx=gxd[b], gy=gyd[b])
            done[b].record(stream)
            with torch.cuda.stream(copy):
                if k + 1 < n_steps:      # next positions, once step k - 1 is done with the buffers
                    if k >= 1:
                        copy.wait_event(done[1 - b])
                    xd[1 - b].copy_(xh[(k + 1) % N_POS_SETS], non_blocking=True)
                    yd[1 - b].copy_(yh[(k + 1) % N_POS_SETS], non_blocking=True)
                    h2d[1 - b].record(copy)
                if k >= 2:
                    d2h[b].synchronize()  # the host has read step k - 2's results
                copy.wait_event(done[b])
                gxh[b].copy_(gxd[b], non_blocking=True)
                gyh[b].copy_(gyd[b], non_blocking=True)
                lossh[b].copy_(lossd[b], non_blocking=True)
                d2h[b].record(copy)
        torch.cuda.synchronize(dev)

    e2e_run(3)
    barrier(world)
    t0 = time.perf_counter()
    e2e_run(e2e_steps)
    t_e2e = reduce_max(time.perf_counter() - t0, world, dev)
    e2e = {"value": world * e2e_steps / t_e2e, "unit": UNIT, "h2d_bytes_per_step": 2 * n * 4,
           "d2h_bytes_per_step": 2 * n * 4 + 8, "steps": e2e_steps,
           "api": "TimingGraph.sta_propagate/extract_critical_paths/attraction_update_pairs/"
                  "attraction_loss_fwd_bwd; positions in from pinned host memory and loss + gradient "
                  "out to pinned host memory every step, on a second stream, double-buffered"}

    stages = None
    if args.stages:
        stages = time_stages(G, xs, ys, T, K, loss_buf, gx, gy, stream, 20)
    ktab = kernel_table(G, step, args.warmup + args.steps, nl, info, (cfg.name, K))
    lonly = loss_only(G, xs, ys, loss_buf, gx, gy, stream)
    lonly_fused = loss_only(G, xs, ys, loss_buf, gx, gy, stream, fused=True)
    ploop = {"every_10_of_500": placement_loop(G, xs, ys, T, K, loss_buf, gx, gy, stream, steps=500, every=10),
             "every_15_of_150": placement_loop(G, xs, ys, T, K, loss_buf, gx, gy, stream, steps=150, every=15)}
    netw = net_weighting(G, xs, ys, T, stream)
    incr = None if args.no_incremental else incremental(G, xs, ys, T, K, mv, stream)
    t1 = table1(G, xs[0], ys[0], T) if not args.no_table1 else None
    fp64 = None if args.no_fp64 else fp64_run(nl, xs, ys, T, K, dev, stream, wns, tns)

    # -------------------------------------------------------------- report --
    result = None
    if rank == 0:
        import json as _json
        peaks = {}
        pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
        if os.path.exists(pp):
            with open(pp) as f:
                peaks = _json.load(f)
        hbm = peaks.get("hbm_gbs")
        peak_src = "of measured" if hbm else "of fallback"
        hbm = hbm or 6400.0
        roof = None
        if prof_n > 0:
            per_launch_ms = prof_ms / prof_n
            kern = args.roofline_kernel
            in_model = kern in MODEL_STEPS
            bytes_ = model_bytes(kern, nl, info) if in_model else own_bytes(kern, nl, info)
            achieved = bytes_ / (per_launch_ms / 1000.0) / 1e9
            roof = {"kernel": kern, "bound": "hbm", "achieved": round(achieved, 1),
                    "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                    "peak_source": peak_src, "traffic": profiled_traffic(kern, (cfg.name, K)),
                    "algorithmic_bytes_per_launch": int(bytes_),
                    "bytes_basis": (f"the method's traffic model, step {MODEL_STEPS[kern]} (per-element "
                                    "figures in bench.model_bytes)") if in_model else "this design's own count",
                    "launch_ms": round(per_launch_ms, 4), "launches": prof_n,
                    "launch_unit": LAUNCH_UNIT.get(kern, "one kernel launch")}
            if kern == "fwd_sweep":
                lb = list_bytes(nl, info)
                ob = own_bytes(kern, nl, info)
                roof["sidetrack_lists"] = {
                    "bytes_per_launch": int(lb), "gbs": round(lb / (per_launch_ms / 1000.0) / 1e9, 1),
                    "note": "top-K search data (a9) built inside the sweep; not counted in achieved"}
                roof["own_bytes_per_launch"] = int(ob)
                roof["own_gbs"] = round(ob / (per_launch_ms / 1000.0) / 1e9, 1)
        cfgd = workload_desc(cfg, nl)
        cfgd.update({"seed": args.seed, "placements": f"{N_POS_SETS} seeded Gaussian moves (sigma {SIGMA} um), cycled",
                     "formed_on_request": "not in the timed iteration, which consumes none of them: required times "
                                          "and slacks of pins other than endpoints, input pins' arrivals "
                                          "(sta_get_timing), the (slack, pin) order of the failing endpoints and "
                                          "the paths' pin lists (sta_get_paths)",
                     "l2": "no flush: per-step working set (netlist + timing state, ~0.5 GB) exceeds the 126 MB L2",
                     "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                     "w0": W0, "w1": W1, "beta": BETA})
        result = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic: seeded levelized random netlist standing in for the ICCAD 2015 superblue designs",
            "config": cfgd, "roofline": roof, "e2e": e2e, "gpu_launches": launches,
            "gpu_launches_per_step": round(launches / args.steps, 1), "clocks": clk,
            "timing": {"wns_ps": wns, "tns_ps": tns, "T_ps": T, "failing_endpoints": n_viol,
                       "paths_per_step": n_paths, "path_pins_per_step": n_path_pins, "pairs_after": n_pairs},
        }
        for v in ktab.values():
            v["own_frac"] = round(v["own_gbs"] / hbm, 4)
        result["kernels"] = ktab
        result["roofline_per_kernel"] = roofline_per_kernel(ktab, nl, info, hbm)
        result["loss_only"] = lonly
        result["loss_only_fused"] = lonly_fused
        result["placement_loop"] = ploop
        result["net_weighting"] = netw
        if incr:
            result["incremental"] = incr
        if stages:
            result["stages_ms"] = stages
        if t1:
            result["table1"] = t1
        if fp64:
            result["fp64_gpu"] = fp64
        if world == 1 and not args.no_cpu_baseline:
            placements = [(xs[k].double().cpu().numpy(), ys[k].double().cpu().numpy()) for k in range(2)]
            ref = {}
            result["cpu_baseline"] = cpu_baseline(nl, cfg, T, placements, keep=ref)
            result["errors_vs_oracle"] = errors_vs_oracle(G, nl, K, T, xs[0], ys[0], ref)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return result


def fp64_run(nl, xs, ys, T, K, dev, stream, wns32, tns32, steps=20):
    """The same timing iteration on an FP64 graph (same kernels in double
    precision): throughput, and the FP32 run's WNS / TNS against it."""
    import torch
    from paper_2503_11674_b300 import TimingGraph
    G = TimingGraph(nl, "fp64", device=dev)
    n = nl.n_cells
    loss = torch.zeros((), dtype=torch.float64, device=dev)
    gx = torch.empty(n, dtype=torch.float64, device=dev)
    gy = torch.empty(n, dtype=torch.float64, device=dev)
    x64, y64 = xs.double(), ys.double()

    def step(k):
        x, y = x64[k % N_POS_SETS], y64[k % N_POS_SETS]
        G.sta_propagate(x, y, T, sync=False)
        G.extract_critical_paths(-1, K, False, sync=False)
        G.attraction_update_pairs(W0, W1, sync=False)
        G.attraction_loss_fwd_bwd(x, y, BETA, out=loss, gx=gx, gy=gy)

    for k in range(3):
        step(k)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        step(3 + k)
    G.sta_join()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    wns64, tns64 = G.sta_propagate(x64[0], y64[0], T)
    del G
    return {"value": round(1000.0 / ms, 2), "unit": UNIT, "ms_per_step": round(ms, 4), "steps": steps,
            "wns_ps": wns64, "tns_ps": tns64,
            "fp32_wns_rel_diff": abs(wns32 - wns64) / max(abs(wns64), 1e-30),
            "fp32_tns_rel_diff": abs(tns32 - tns64) / max(abs(tns64), 1e-30)}


def time_stages(G, xs, ys, T, K, loss_buf, gx, gy, stream, reps):
    """Device time of each entry point, bracketed by events (diagnostic)."""
    import torch
    names = ["sta_propagate", "extract_critical_paths", "attraction_update_pairs",
             "attraction_loss_fwd", "attraction_loss_bwd"]
    tot = {k: 0.0 for k in names}
    for r in range(reps):
        x, y = xs[r % len(xs)], ys[r % len(ys)]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        ev[0].record(stream)
        G.sta_propagate(x, y, T, sync=False)
        G.sta_join()  # the whole STA, backward sweep included
        ev[1].record(stream)
        G.extract_critical_paths(-1, K, False, sync=False)
        ev[2].record(stream)
        G.attraction_update_pairs(W0, W1, sync=False)
        ev[3].record(stream)
        G.attraction_loss_fwd(x, y, BETA, out=loss_buf)
        ev[4].record(stream)
        G.attraction_loss_bwd(x, y, BETA, gx=gx, gy=gy)
        ev[5].record(stream)
        torch.cuda.synchronize()
        for i, k in enumerate(names):
            tot[k] += ev[i].elapsed_time(ev[i + 1])
    out = {k: round(v / reps, 4) for k, v in tot.items()}
    # the loss variants of the ablation (same pair set, same placement)
    kinds = {}
    for kind in ("quadratic", "hpwl", "euclid"):
        G.attraction_set_loss_kind(kind)
        f = b = 0.0
        for r in range(reps):
            x, y = xs[r % len(xs)], ys[r % len(ys)]
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            G.attraction_loss_fwd(x, y, BETA, out=loss_buf)
            ev[1].record(stream)
            G.attraction_loss_bwd(x, y, BETA, gx=gx, gy=gy)
            ev[2].record(stream)
            torch.cuda.synchronize()
            f += ev[0].elapsed_time(ev[1])
            b += ev[1].elapsed_time(ev[2])
        kinds[kind] = {"fwd_ms": round(f / reps, 4), "bwd_ms": round(b / reps, 4)}
    G.attraction_set_loss_kind("quadratic")
    out["loss_kinds"] = kinds
    return out


KERNEL_TABLE = ["net_rc", "fwd_sweep", "ep_wns", "bwd_sweep", "topk", "pair_walk", "pp_fwd_bwd", "pp_bwd_cell"]


def kernel_table(G, step, k0, nl, info, workload, reps=10):
    """Live duration of every kernel of the iteration in the steady state (CUDA
    events on the kernel's own stream, one kernel at a time), its algorithmic
    bytes and the GB/s they make.  The backward sweep runs beside extraction,
    the pair update and the loss, on its share of the SMs."""
    import torch
    out = {}
    for name in KERNEL_TABLE:
        G.tdp_profile_kernel(name)
        for k in range(reps):
            step(k0 + k)
        G.sta_join()
        torch.cuda.synchronize()
        n, ms = G.tdp_profile_read()
        G.tdp_profile_kernel(None)
        if n == 0:
            continue
        per = ms / n
        by = own_bytes(name, nl, info)
        out[name] = {"ms": round(per, 4), "own_bytes": int(by), "own_gbs": round(by / (per / 1e3) / 1e9, 1)}
        tr = profiled_traffic(name, workload)
        if tr is not None:
            out[name]["dram_traffic"] = tr
            out[name]["dram_gbs"] = round(tr / (per / 1e3) / 1e9, 1)
    return out


def roofline_per_kernel(ktab, nl, info, hbm):
    """Each propagation, extraction and loss kernel against the measured HBM
    peak, by the method's traffic model (model_bytes) and its live duration
    from kernel_table.  The search and the pair walk together do a7-a10; the
    two backward loss kernels together a11's backward pass."""
    rows = {}

    def add(step, ms, kernels):
        b = model_bytes(step, nl, info)
        g = b / (ms / 1e3) / 1e9
        rows[step] = {"step": MODEL_STEPS[step], "kernels": kernels, "ms": round(ms, 4), "model_bytes": int(b),
                      "gbs": round(g, 1), "frac": round(g / hbm, 4)}

    for k in ("net_rc", "fwd_sweep", "bwd_sweep", "ep_wns"):
        if k in ktab:
            add(k, ktab[k]["ms"], [k])
    if "topk" in ktab and "pair_walk" in ktab:
        add("topk+pair_walk", ktab["topk"]["ms"] + ktab["pair_walk"]["ms"], ["topk", "pair_walk"])
    if "pp_fwd_bwd" in ktab and "pp_bwd_cell" in ktab:
        add("pp_fwd_bwd", ktab["pp_fwd_bwd"]["ms"] + ktab["pp_bwd_cell"]["ms"], ["pp_fwd_bwd", "pp_bwd_cell"])
    return rows


def loss_step(G, x, y, loss_buf, gx, gy, fused):
    """The loss and its gradient: two calls (attraction_loss_fwd, _bwd) or the
    fused one (attraction_loss_fwd_bwd, the same bits in two launches)."""
    if fused:
        G.attraction_loss_fwd_bwd(x, y, BETA, out=loss_buf, gx=gx, gy=gy)
    else:
        G.attraction_loss_fwd(x, y, BETA, out=loss_buf)
        G.attraction_loss_bwd(x, y, BETA, gx=gx, gy=gy)


def loss_only(G, xs, ys, loss_buf, gx, gy, stream, steps=100, fused=False):
    """Steps of the attraction loss alone (forward + backward) on the current
    pair set, as a placement step between two timing iterations runs it."""
    import torch
    def one(k):
        loss_step(G, xs[k % len(xs)], ys[k % len(ys)], loss_buf, gx, gy, fused)
    for k in range(5):
        one(k)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        one(k)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return {"value": round(1000.0 / ms, 1), "unit": "loss fwd+bwd steps/s", "ms_per_step": round(ms, 4),
            "call": "attraction_loss_fwd_bwd" if fused else "attraction_loss_fwd + attraction_loss_bwd"}


def placement_loop(G, xs, ys, T, K, loss_buf, gx, gy, stream, steps=150, every=15, fused=True):
    """The hot path as placement uses it: the loss forward + backward every
    step, a timing iteration (STA, extraction, pair update) every `every`
    steps.  The 1.2M-cell workload is configured as one timing iteration
    every 10 steps of a 500-step loop; the paper re-times every m = 15 steps
    (Section IV)."""
    import torch
    def one(k):
        x, y = xs[k % len(xs)], ys[k % len(ys)]
        if k % every == 0:
            G.sta_propagate(x, y, T, sync=False)
            G.extract_critical_paths(-1, K, False, sync=False)
            G.attraction_update_pairs(W0, W1, sync=False)
        loss_step(G, x, y, loss_buf, gx, gy, fused)
    for k in range(every):
        one(k)
    G.sta_join()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        one(k)
    G.sta_join()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return {"value": round(1000.0 / ms, 1), "unit": "placement steps/s", "steps": steps, "timing_every": every,
            "ms_per_step": round(ms, 4),
            "loss_call": "attraction_loss_fwd_bwd" if fused else "attraction_loss_fwd + attraction_loss_bwd"}


def net_weighting(G, xs, ys, T, stream, alpha=0.5, gamma=4.0, steps=20):
    """The net-weighting baseline's timing iteration on this workload (the
    "w/o Path Extraction" scheme): a full STA, whose backward sweep's
    required times the weights need, and one momentum update of every net's
    weight from its worst pin slack (net_weights_update).  Also the update
    kernel alone: 28 B per net (net pointer, required-time key, driver
    arrival, weight read and written)."""
    import torch
    G.net_weights_reset()

    def one(k):
        G.sta_propagate(xs[k % len(xs)], ys[k % len(ys)], T, sync=False)
        G.net_weights_update(alpha, gamma, sync=False)

    for k in range(3):
        one(k)
    G.sta_join()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    G.tdp_profile_kernel("net_weights")
    e0.record(stream)
    for k in range(steps):
        one(3 + k)
    G.sta_join()
    e1.record(stream)
    torch.cuda.synchronize()
    n, kms = G.tdp_profile_read()
    G.tdp_profile_kernel(None)
    ms = e0.elapsed_time(e1) / steps
    n_crit = G.net_weights_update(alpha, gamma)
    by = 28.0 * G.n_nets
    per = kms / max(n, 1)
    return {"value": round(1000.0 / ms, 1), "unit": "iter/s", "ms_per_step": round(ms, 4), "steps": steps,
            "alpha": alpha, "gamma": gamma, "critical_nets": n_crit,
            "update_kernel": {"ms": round(per, 4), "bytes": int(by), "gbs": round(by / (per / 1e3) / 1e9, 1)}}


INC_MOVED = (1, 12, 120, 1200, 12000, 120000, None)  # cells moved per call; None: every movable cell


def incremental(G, xs, ys, T, K, mv, stream, reps=20):
    """Incremental timing (sta_propagate_incremental) on this workload.  For
    each number of moved cells, calls alternate between a placement and the
    same with that many movable cells moved (seeded Gaussian, sigma as the
    placements), so that every call sees that many moves.  Per call (median
    of `reps`, CUDA events on the library stream): the graph's stream until
    WNS / TNS are ready, the same with the backward sweep joined, and a whole
    timing iteration (incremental STA, extraction, pair update, loss);
    beside them the full sta_propagate, and what the library re-evaluated."""
    import torch
    dev = xs.device
    n = xs.shape[1]
    gen = torch.Generator(device=dev)
    gen.manual_seed(77)
    movable = torch.nonzero(mv).flatten()
    x0, y0 = xs[0].clone(), ys[0].clone()
    buf = torch.zeros((), dtype=torch.float64, device=dev)
    gx = torch.empty(n, dtype=torch.float32, device=dev)
    gy = torch.empty(n, dtype=torch.float32, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def med(v):
        return round(sorted(v)[len(v) // 2], 4)

    def measure(prop, pos):
        for r in range(2):
            prop(*pos[(r + 1) % 2], T, sync=False)
        G.sta_join()
        t_main, t_all, t_it = [], [], []
        for r in range(2 * reps):
            x, y = pos[(r + 1) % 2]
            torch.cuda.synchronize()
            ev[0].record(stream)
            prop(x, y, T, sync=False)
            ev[1].record(stream)
            if r < reps:
                G.sta_join()
            else:
                G.extract_critical_paths(-1, K, False, sync=False)
                G.attraction_update_pairs(W0, W1, sync=False)
                G.attraction_loss_fwd_bwd(x, y, BETA, out=buf, gx=gx, gy=gy)
                G.sta_join()
            ev[2].record(stream)
            torch.cuda.synchronize()
            if r < reps:
                t_main.append(ev[0].elapsed_time(ev[1]))
                t_all.append(ev[0].elapsed_time(ev[2]))
            else:
                t_it.append(ev[0].elapsed_time(ev[2]))
        return {"propagate_ms": med(t_main), "propagate_with_bwd_ms": med(t_all), "iteration_ms": med(t_it)}

    G.sta_propagate_incremental(x0, y0, T)
    G.extract_critical_paths(-1, K, False)  # sidetrack lists of the iteration's length
    rows = []
    for m in INC_MOVED:
        if m is None:
            x1, y1 = xs[1], ys[1]
        else:
            idx = movable[torch.randperm(movable.numel(), generator=gen, device=dev)[:m]]
            x1, y1 = x0.clone(), y0.clone()
            x1[idx] += SIGMA * torch.randn(m, generator=gen, device=dev)
            y1[idx] += SIGMA * torch.randn(m, generator=gen, device=dev)
        row = {"moved_cells": m if m is not None else int(movable.numel())}
        row.update(measure(G.sta_propagate_incremental, [(x0, y0), (x1, y1)]))
        st = G.incremental_stats()
        row.update({"cells_evaluated_selectively": st["cells_evaluated"], "cells_changed": st["cells_changed"],
                    "levels": [st["first_level"], st["last_level"]],
                    "every_cell_from_level": st["every_cell_from_level"], "fell_back_to_full": bool(st["full"])})
        rows.append(row)
    full = measure(G.sta_propagate, [(x0, y0), (xs[1], ys[1])])
    return {"unit": "ms per call", "K": K, "rows": rows, "full_sta_propagate": full}


def table1(G, x, y, T, reps=3):
    """Table I's comparison on this workload: report_timing(n) with n = the
    failing endpoints and 10 n, against report_timing_endpoint(n, 1) and
    (n, 10).  Per command: paths, distinct endpoints, distinct pin pairs (the
    pair set after one update from an empty set), and the time of the call
    (median of `reps`, synchronised on both sides)."""
    import torch
    G.sta_propagate(x, y, T)
    G.extract_critical_paths(-1, 1, False)
    nv = G.sta_get_paths_size()[0]
    cmds = [(f"report_timing({nv})", lambda: G.report_timing(nv), True),
            (f"report_timing({10 * nv})", lambda: G.report_timing(10 * nv), True),
            (f"report_timing_endpoint({nv},1)", lambda: G.extract_critical_paths(nv, 1, False), False),
            (f"report_timing_endpoint({nv},10)", lambda: G.extract_critical_paths(nv, 10, False), False)]
    rows = []
    for name, fn, global_search in cmds:
        times, n_paths, exp_ms = [], 0, None
        for r in range(reps):
            if global_search and r == reps - 1:
                G.tdp_profile_kernel("rt_expand")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            n_paths = fn()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
            if global_search and r == reps - 1:
                exp_ms = G.tdp_profile_read()
                G.tdp_profile_kernel(None)
        P = G.sta_get_paths()
        n_ep = int(torch.unique(P["ep"]).numel())
        G.attraction_reset_pairs()
        n_pairs = G.attraction_update_pairs(W0, W1)
        row = {"command": name, "paths": int(n_paths), "endpoints": n_ep, "pin_pairs": int(n_pairs),
               "ms": round(1e3 * sorted(times)[len(times) // 2], 3)}
        if exp_ms is not None:
            row["rt_expand"] = {"launches": exp_ms[0], "ms": round(exp_ms[1], 3)}
        rows.append(row)
    G.attraction_reset_pairs()
    return {"failing_endpoints": int(nv), "rows": rows}


# ------------------------------------------------------------ CPU oracle --

def oracle_iteration(nl, cfg, T, pos, state=None, keep=None):
    """One full timing iteration of the FP64 oracle at placement `pos`: STA of
    the whole netlist, report_timing_endpoint(all failing endpoints, K) in
    one call, the Eq. (w_ij) pair update (the pair set `state` carried from
    the last iteration) and the loss.  Returns its seconds, the new state and
    the number of failing endpoints; with `keep` (a dict) it also leaves the
    timing, the paths and the new pair set there."""
    import oracle
    x, y = pos
    t0 = time.perf_counter()
    tm = oracle.sta(nl, x, y, T)
    P = oracle.topk(nl, tm, -1, cfg.K)
    in_p, w = oracle.update_pairs(nl, P, tm["wns"], W0, W1,
                                  None if state is None else state[0], None if state is None else state[1])
    oracle.loss(nl, in_p, w, BETA, x, y)
    sec = time.perf_counter() - t0
    if keep is not None:
        keep.update(tm=tm, paths=P, in_p=in_p, w=w)
    return sec, (in_p, w), len(P["viol"])


def host_cpu() -> dict:
    """The host's CPU: logical cores (nproc), those this process may use, and the model."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "usable": len(os.sched_getaffinity(0)), "model": model}


def cpu_baseline(nl, cfg, T, placements, keep=None):
    """The oracle as it stands on one host core: full timing iterations (every
    failing endpoint, nothing scaled) at consecutive placements, the pair set
    carried from one to the next as in the placement loop.  `keep` receives
    the first iteration's results (for the error report)."""
    state, total, nvs = None, 0.0, []
    for i, pos in enumerate(placements):
        sec, state, nv = oracle_iteration(nl, cfg, T, pos, state, keep if i == 0 else None)
        total += sec
        nvs.append(nv)
    n = len(placements)
    return {"value": round(n / total, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "host": host_cpu(),
            "sample": f"{n} full timing iterations of the same workload at consecutive placements: FP64 STA, "
                      f"top-{cfg.K} extraction on every failing endpoint ({', '.join(str(v) for v in nvs)}), "
                      f"pair update and loss; {total:.1f} s of single-threaded CPU work",
            "seconds_per_iteration": round(total / n, 3)}


def errors_vs_oracle(G, nl, K, T, xd, yd, ref):
    """The FP32 GPU results at one placement against the FP64 oracle's at the
    same placement (the first CPU-baseline iteration, `ref`), per result:
    arrival, required time and slack of every pin (max |d| in ps, max |d| /
    value scale, and max |d| over the stated tolerance 1e-3 ps + 1e-6 x
    scale: at most 1 is within it); WNS / TNS relative; the path sets of every
    failing endpoint under the margin rule (decided endpoints must match
    exactly); the pair set after one update from an empty set; the loss and
    the gradient on the GPU's pair set (relative, relative L2)."""
    import numpy as np
    tests_dir = os.path.join(ROOT, "tests")
    if tests_dir not in sys.path:
        sys.path.insert(0, tests_dir)
    import oracle
    from parity_util import TOL32, compare_paths, sta_scales
    tm = ref["tm"]
    a, r = TOL32
    out = {"tolerance": "|d| <= 1e-3 ps + 1e-6 x scale; scale: |arr|, max(|req|, T - req), "
                        "max(|arr|, |req|, T - slack)"}
    wns, tns = G.sta_propagate(xd, yd, T)
    got = [t.double().cpu().numpy() for t in G.sta_get_timing()]
    for name, g, sc in zip(("arr", "req", "slack"), got, sta_scales(tm, T)):
        d = np.abs(g - tm[name])
        out[name] = {"max_abs_ps": float(d.max()),
                     "max_rel": float((d / np.maximum(np.abs(sc), 1e-30)).max()),
                     "max_over_tol": float((d / (a + r * np.abs(sc))).max())}
    out["wns_rel"] = abs(wns - tm["wns"]) / max(abs(tm["wns"]), 1e-30)
    out["tns_rel"] = abs(tns - tm["tns"]) / max(abs(tm["tns"]), 1e-30)
    G.extract_critical_paths(-1, K, False)
    P = {k: v.cpu().numpy() for k, v in G.sta_get_paths().items()}
    try:
        d = compare_paths(nl, tm, T, K, False, P, TOL32, detail=True)
        out["paths"] = {"decided_endpoints": d["checked"], "decided_mismatching": 0,
                        "ambiguous_endpoints": d["ambiguous"], "ambiguous_with_another_set": len(d["differ"]),
                        "paths": d["paths"], "max_slack_abs_ps": float(d["max_slack_err"])}
    except AssertionError as e:
        out["paths"] = {"decided_mismatching": "at least 1", "first_failure": str(e)[:300]}
    G.attraction_reset_pairs()
    G.attraction_update_pairs(W0, W1)
    pins, w = G.attraction_get_pairs()
    pins, w = pins.cpu().numpy().astype(np.int64), w.double().cpu().numpy()
    in_ref, w_ref = oracle.update_pairs(nl, ref["paths"], tm["wns"], W0, W1)
    ref_pins = np.nonzero(in_ref)[0]
    common = np.intersect1d(pins, ref_pins)
    wg = np.zeros(nl.n_pins)
    wg[pins] = w
    out["pairs"] = {"gpu": int(len(pins)), "oracle": int(len(ref_pins)),
                    "symmetric_difference": int(len(np.setxor1d(pins, ref_pins))),
                    "max_rel_weight_diff": float((np.abs(wg[common] - w_ref[common]) /
                                                  np.abs(w_ref[common])).max()) if len(common) else 0.0}
    in_p = np.zeros(nl.n_pins, np.uint8)
    in_p[pins] = 1
    x0, y0 = xd.double().cpu().numpy(), yd.double().cpu().numpy()
    pp, gx_r, gy_r = oracle.loss(nl, in_p, wg, BETA, x0, y0)
    lg = G.attraction_loss_fwd(xd, yd, BETA).item()
    gx, gy = G.attraction_loss_bwd(xd, yd, BETA)
    g = np.concatenate([gx.double().cpu().numpy(), gy.double().cpu().numpy()])
    gr = np.concatenate([gx_r, gy_r])
    out["loss_rel"] = abs(lg - pp) / max(abs(pp), 1e-30)
    out["grad_rel_l2"] = float(np.linalg.norm(g - gr) / max(np.linalg.norm(gr), 1e-30))
    return out


REF_BUDGET_S = 150.0  # timed oracle work of the reference arm at most (its run ends within minutes)


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on one host core.  A
    step is one full timing iteration at a new placement (oracle_iteration,
    nothing sampled or scaled; about 7 s at 1.2M cells), after one warm-up
    iteration.  The timed steps stop at K or once REF_BUDGET_S of them have
    run (at least two), so that the run ends within minutes; the line says
    how many were timed."""
    import netgen
    world, rank, _ = dist_env()
    if rank != 0:
        return None
    cfg = netgen.CONFIGS[args.config]
    if args.K:
        import dataclasses
        cfg = dataclasses.replace(cfg, K=args.K)
    nl = netgen.generate(cfg, args.seed)
    import numpy as np
    import oracle
    rng = np.random.default_rng(1000 + args.seed)
    x, y = nl.x.astype(np.float64), nl.y.astype(np.float64)
    mv = nl.cell_fixed == 0
    T = oracle.clock_period(nl, cfg.t_factor, x, y)

    def placement():
        nonlocal x, y
        x = np.where(mv, np.clip(x + rng.normal(0, SIGMA, len(x)), 0, netgen.DIE_UM), x)
        y = np.where(mv, np.clip(y + rng.normal(0, SIGMA, len(y)), 0, netgen.DIE_UM), y)
        return x, y

    state = None
    warm = min(args.warmup, 1)
    for _ in range(warm):
        _, state, _ = oracle_iteration(nl, cfg, T, placement(), state)
    times = []
    while len(times) < args.steps and (len(times) < 2 or sum(times) < REF_BUDGET_S):
        sec, state, nv = oracle_iteration(nl, cfg, T, placement(), state)
        times.append(sec)
    value = len(times) / sum(times)
    cfgd = workload_desc(cfg, nl)
    cfgd.update({"seed": args.seed, "parallelism": "single CPU thread"})
    sample = (f"each step one full timing iteration at a new placement: FP64 STA of the whole netlist, "
              f"top-{cfg.K} extraction on every failing endpoint ({nv} at the last), pair update, loss; "
              f"{len(times)} of {args.steps} steps timed ({sum(times):.1f} s; the timed steps stop at "
              f"{REF_BUDGET_S:.0f} s), {warm} warm-up iteration")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "steps_timed": len(times), "warmup": args.warmup, "warmup_run": warm,
            "ms_per_step": round(1000.0 / value, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic: seeded levelized random netlist standing in for the ICCAD 2015 superblue designs",
            "config": cfgd,
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample, "cpu_seconds": round(sum(times), 1)},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse_args()
    res = run_reference(args) if args.impl == "reference" else run_ours(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
