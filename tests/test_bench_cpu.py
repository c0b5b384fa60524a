"""bench.py's CPU paths, on a small netlist: the reference arm (the oracle as
it stands, one full timing iteration a step) and the CPU baseline."""
import numpy as np

import bench
import netgen
import oracle


class _Args:
    config, seed, steps, warmup, K = "tiny", 1, 3, 2, None


def _single_rank(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)


def test_reference_arm_line(monkeypatch):
    _single_rank(monkeypatch)
    r = bench.run_reference(_Args())
    assert r["impl"] == "reference" and r["metric"] == bench.METRIC and r["unit"] == bench.UNIT
    assert r["higher_is_better"] is True and r["value"] > 0
    assert (r["steps"], r["steps_timed"], r["warmup"], r["warmup_run"]) == (3, 3, 2, 1)
    assert r["e2e"] == {"value": r["value"], "unit": r["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == r["value"]
    assert r["ms_per_step"] == round(1000.0 / r["value"], 1)


def test_reference_arm_stops_its_timed_steps_at_the_budget(monkeypatch):
    _single_rank(monkeypatch)
    monkeypatch.setattr(bench, "REF_BUDGET_S", 0.0)

    class Args(_Args):
        steps = 50

    r = bench.run_reference(Args())
    assert r["steps"] == 50 and r["steps_timed"] == 2  # at least two, then the budget ends them


def test_cpu_baseline_times_full_iterations():
    cfg = netgen.CONFIGS["tiny"]
    nl = netgen.generate(cfg, 1)
    T = oracle.clock_period(nl, cfg.t_factor)
    x2, y2 = netgen.perturb(nl.x, nl.y, nl.cell_fixed, 2.0, np.random.default_rng(0))
    cb = bench.cpu_baseline(nl, cfg, T, [(nl.x, nl.y), (x2, y2)])
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] > 0
    assert cb["sample"].startswith("2 full timing iterations")
    assert abs(cb["seconds_per_iteration"] - 1.0 / cb["value"]) < 1e-3


def test_cpu_baseline_keeps_the_first_iteration_and_names_the_host():
    cfg = netgen.CONFIGS["tiny"]
    nl = netgen.generate(cfg, 1)
    T = oracle.clock_period(nl, cfg.t_factor)
    keep = {}
    cb = bench.cpu_baseline(nl, cfg, T, [(nl.x, nl.y)], keep=keep)
    assert set(keep) == {"tm", "paths", "in_p", "w"}
    assert keep["tm"]["T"] == T and len(keep["paths"]["viol"]) > 0
    assert cb["host"]["nproc"] >= 1 and 1 <= cb["host"]["usable"] <= cb["host"]["nproc"]


def test_model_bytes_follow_the_per_element_figures():
    nl = netgen.generate("tiny", 1)
    c = bench.netlist_counts(nl)
    assert c["sinks"] == nl.n_pins - nl.n_nets
    assert c["comb_inputs"] + c["endpoints"] == c["sinks"]
    info = {"path_pins": 1000, "pairs": 50, "list_L": 15}
    assert bench.model_bytes("fwd_sweep", nl, info) == 16 * c["comb_inputs"] + 16 * c["comb"] + 4 * nl.n_pins
    assert bench.model_bytes("net_rc", nl, info) == 32 * (c["sinks"] + nl.n_nets)
    assert bench.model_bytes("bwd_sweep", nl, info) == 12 * nl.n_pins
    assert bench.model_bytes("topk+pair_walk", nl, info) == 52 * 500
    assert bench.model_bytes("pp_fwd_bwd", nl, info) == 80 * 50 + 8 * nl.n_pins + 8 * nl.n_cells
    assert bench.list_bytes(nl, info) == c["comb"] * 16 * 15
    assert set(bench.MODEL_STEPS) == {"net_rc", "fwd_sweep", "bwd_sweep", "ep_wns", "topk+pair_walk",
                                      "pp_fwd_bwd"}
