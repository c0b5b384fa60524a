"""Incremental timing (sta_propagate_incremental) through the C ABI.

Its results are those of a full propagation bit for bit, for every kind of
move (none, one cell, a fraction of the cells, every cell, cells moved back,
a new clock period), with and without sidetrack lists, in FP32 and FP64; its
forward sweep re-evaluates only cells in the structural fan-out cone of the
moved cells; and it agrees with the FP64 oracle at the end of a sequence.
"""
import numpy as np
import pytest
import torch

import netgen
import oracle
from parity_util import check_sta, gpu_paths, tol_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2503_11674_b300.build import build
    build()


def _graph(nl, prec):
    from paper_2503_11674_b300 import TimingGraph
    return TimingGraph(nl, prec)


def _t(a, dtype):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def _assert_same_state(A, B):
    for a, b in zip(A.sta_get_timing() + A.sta_get_net_delays(), B.sta_get_timing() + B.sta_get_net_delays()):
        assert torch.equal(a, b)


def _assert_same_paths(A, B, K):
    assert A.extract_critical_paths(-1, K) == B.extract_critical_paths(-1, K)
    Pa, Pb = gpu_paths(A), gpu_paths(B)
    assert Pa.keys() == Pb.keys()
    for k in Pa:
        np.testing.assert_array_equal(Pa[k], Pb[k])


def _moves(nl, rng):
    """Position sets, each differing from the one before by the named move."""
    seq = [("initial", nl.x, nl.y), ("none", nl.x.copy(), nl.y.copy())]
    comb = np.nonzero(nl.cell_type == netgen.COMB)[0]
    x, y = nl.x.copy(), nl.y.copy()
    x[int(rng.choice(comb))] += np.float32(3.0)
    seq.append(("one cell", x, y))
    for frac in (0.001, 0.01, 0.1):
        x, y = seq[-1][1].copy(), seq[-1][2].copy()
        idx = rng.choice(nl.n_cells, max(1, int(frac * nl.n_cells)), replace=False)
        x[idx] += rng.normal(0.0, 2.0, len(idx)).astype(np.float32)
        y[idx] += rng.normal(0.0, 2.0, len(idx)).astype(np.float32)
        seq.append((f"{frac:g} of the cells", x, y))
    x, y = netgen.perturb(seq[-1][1], seq[-1][2], nl.cell_fixed, 2.0, rng)
    seq.append(("every cell", x, y))
    seq.append(("back to an earlier placement", seq[3][1], seq[3][2]))
    return seq


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("cfg,K", [("tiny", 0), ("tiny", 4), ("mid", 16), ("mid", 32)])
def test_incremental_matches_full_propagation(cfg, K, prec):
    nl = netgen.generate(cfg, 3)
    T = oracle.clock_period(nl, netgen.CONFIGS[cfg].t_factor)
    A, B = _graph(nl, prec), _graph(nl, prec)  # A incremental, B full
    rng = np.random.default_rng(7)
    seq = _moves(nl, rng)
    seen_sat = False
    for i, (name, x, y) in enumerate(seq):
        xa, ya = _t(x, A.dtype), _t(y, A.dtype)
        assert A.sta_propagate_incremental(xa, ya, T) == B.sta_propagate(xa, ya, T), name
        st = A.incremental_stats()
        assert st["full"] == (1 if i == 0 else 0), (name, st)
        if name == "none":
            assert (st["moved_cells"], st["cells_evaluated"], st["last_level"]) == (0, 0, -1), st
        if name == "one cell":
            assert st["moved_cells"] == 1 and st["cells_changed"] <= st["cells_evaluated"], st
        seen_sat = seen_sat or st["every_cell_from_level"] > 0
        _assert_same_state(A, B)
        if K:
            _assert_same_paths(A, B, K)
    assert seen_sat  # moving every cell saturates: both parts of the sweep are exercised
    # a new clock period and no move: required times and slacks change only
    T2 = 0.9 * T
    assert A.sta_propagate_incremental(xa, ya, T2) == B.sta_propagate(xa, ya, T2)
    assert A.incremental_stats()["cells_evaluated"] == 0
    _assert_same_state(A, B)
    # and the oracle at the last placement
    tm = oracle.sta(nl, np.asarray(seq[-1][1], np.float64), np.asarray(seq[-1][2], np.float64), T2)
    check_sta(A, tm, T2, tol_of(A.dtype))


def _fanout_cone(nl, cells):
    """Combinational cells whose inputs or delay a move of `cells` can reach:
    the drivers and sinks of their nets, and everything downstream."""
    pin_net = np.repeat(np.arange(nl.n_nets), np.diff(nl.net_ptr))
    comb = nl.cell_type == netgen.COMB
    out_net = np.full(nl.n_cells, -1)
    drv = nl.net_ptr[:-1]
    out_net[nl.pin_cell[drv]] = np.arange(nl.n_nets)
    sinks = [nl.pin_cell[nl.net_ptr[e] + 1:nl.net_ptr[e + 1]] for e in range(nl.n_nets)]
    nets = set(pin_net[np.isin(nl.pin_cell, cells)].tolist())
    cone, todo = set(), []
    for e in nets:
        for c in [int(nl.pin_cell[drv[e]])] + sinks[e].tolist():
            if comb[c] and c not in cone:
                cone.add(c)
                todo.append(c)
    while todo:
        c = todo.pop()
        for s in sinks[out_net[c]].tolist():
            if comb[s] and s not in cone:
                cone.add(s)
                todo.append(s)
    return cone


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_incremental_sweep_stays_in_the_fanout_cone(seed):
    nl = netgen.generate("diff", seed)
    T = oracle.clock_period(nl, 0.9)
    G = _graph(nl, "fp32")
    G.sta_propagate_incremental(_t(nl.x, G.dtype), _t(nl.y, G.dtype), T)
    G.extract_critical_paths(-1, 8)
    rng = np.random.default_rng(seed)
    comb = np.nonzero(nl.cell_type == netgen.COMB)[0]
    x, y = nl.x.copy(), nl.y.copy()
    for n_moved in (1, 1, 5, 50):
        cells = rng.choice(comb, n_moved, replace=False)
        x[cells] += rng.normal(0.0, 5.0, n_moved).astype(np.float32)
        G.sta_propagate_incremental(_t(x, G.dtype), _t(y, G.dtype), T)
        st = G.incremental_stats()
        cone = _fanout_cone(nl, cells)
        assert st["moved_cells"] == n_moved
        # selective evaluation stays in the cone (and, past the level where the
        # changes saturate, every cell is evaluated without checks)
        assert 0 < st["cells_evaluated"] <= len(cone), (st, len(cone))
        assert st["cells_changed"] <= st["cells_evaluated"]
        assert 1 <= st["first_level"] <= st["last_level"] <= nl.meta["config"]["depth"], st
        sat = st["every_cell_from_level"]
        assert sat == 0 or (st["first_level"] < sat and st["last_level"] == nl.meta["config"]["depth"]), st


def test_full_propagation_keeps_positions_for_the_next_incremental_call():
    nl = netgen.generate("tiny", 5)
    T = oracle.clock_period(nl, 0.9)
    A, B = _graph(nl, "fp32"), _graph(nl, "fp32")
    x, y = _t(nl.x, A.dtype), _t(nl.y, A.dtype)
    A.sta_propagate_incremental(x, y, T)   # first call: everything, buffers allocated
    x2 = x.clone()
    x2[7] += 1.0
    A.sta_propagate(x2, y, T)              # full, and keeps x2
    assert A.incremental_stats()["full"] == 1
    x3 = x2.clone()
    x3[11] -= 2.0
    B.sta_propagate(x3, y, T)
    assert A.sta_propagate_incremental(x3, y, T) == B.sta_propagate(x3, y, T)
    assert A.incremental_stats()["moved_cells"] == 1
    _assert_same_state(A, B)


def test_level_launch_fallback_re_times_everything(monkeypatch):
    """Where the sweeps run as one launch per level, an incremental call
    re-times everything, with the same results."""
    monkeypatch.setenv("TDP_LEVEL_GRAPHS", "1")
    nl = netgen.generate("tiny", 4)
    T = oracle.clock_period(nl, 0.9)
    A = _graph(nl, "fp32")
    monkeypatch.delenv("TDP_LEVEL_GRAPHS")
    B = _graph(nl, "fp32")
    x, y = _t(nl.x, A.dtype), _t(nl.y, A.dtype)
    A.sta_propagate_incremental(x, y, T)
    x2 = x.clone()
    x2[3] += 1.0
    assert A.sta_propagate_incremental(x2, y, T) == B.sta_propagate(x2, y, T)
    assert A.incremental_stats()["full"] == 1
    _assert_same_state(A, B)


def test_incremental_matches_full_propagation_at_1_2m_cells():
    """The benchmark's workload (1.2M cells, K = 16 lists): 1, 120 and 12,000
    moved cells, each call checked bit for bit against a full propagation,
    timing and paths (the selective sweep, and its hand-over to the full
    sweep once the changes saturate)."""
    cfg = netgen.CONFIGS["1.2M"]
    nl = netgen.generate(cfg, 1)
    T = oracle.clock_period(nl, cfg.t_factor)
    A, B = _graph(nl, "fp32"), _graph(nl, "fp32")
    x, y = nl.x.copy(), nl.y.copy()
    A.sta_propagate_incremental(_t(x, A.dtype), _t(y, A.dtype), T)
    A.extract_critical_paths(-1, cfg.K)  # lists of the iteration's length from here on
    rng = np.random.default_rng(11)
    movable = np.nonzero(nl.cell_fixed == 0)[0]
    seen = []
    for m in (1, 120, 12000):
        idx = rng.choice(movable, m, replace=False)
        x[idx] += rng.normal(0.0, 2.0, m).astype(np.float32)
        y[idx] += rng.normal(0.0, 2.0, m).astype(np.float32)
        xa, ya = _t(x, A.dtype), _t(y, A.dtype)
        assert A.sta_propagate_incremental(xa, ya, T) == B.sta_propagate(xa, ya, T), m
        st = A.incremental_stats()
        assert st["full"] == 0 and st["moved_cells"] == m, st
        seen.append(st["every_cell_from_level"])
        _assert_same_state(A, B)
        _assert_same_paths(A, B, cfg.K)
    assert seen[-1] > 0  # 12,000 moved cells saturate: the full sweep finished the call
