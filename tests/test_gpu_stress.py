"""Parity at the stress size: 3M movable cells (3.3M nets, ~10.5M pins), depth
120, clock at 0.8x the largest arrival, K = 32 paths per failing endpoint.

* STA on every pin and WNS / TNS against the FP64 oracle.
* The extraction of all failing endpoints with K = 32 (the call of a timing
  iteration; ~61,000 endpoints, ~1.9M paths, ~440M path pins) is compared
  with the oracle on every failing endpoint: bit-exact pin sequences on every
  endpoint whose top-K set is decided by more than the slack tolerance, the
  unique part and the validity of every path on the others.  A second
  extraction gives the same bits.
* The pair update runs on the full path set; the loss and its gradient are
  checked with a seeded pair set.
"""
import numpy as np
import pytest
import torch

import netgen
import oracle
from parity_util import TOL32, check_sta, compare_paths

pytestmark = pytest.mark.gpu

CFG = "stress"


@pytest.fixture(scope="module")
def run():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2503_11674_b300 import TimingGraph
    from paper_2503_11674_b300.build import build
    build()
    cfg = netgen.CONFIGS[CFG]
    nl = netgen.generate(CFG, 1)
    T = oracle.clock_period(nl, cfg.t_factor)
    tm = oracle.sta(nl, T=T)
    G = TimingGraph(nl, "fp32")
    x = torch.tensor(nl.x, device="cuda")
    y = torch.tensor(nl.y, device="cuda")
    wns, tns = G.sta_propagate(x, y, T)
    n1 = G.extract_critical_paths(-1, cfg.K, False)
    tot1 = G.sta_get_paths_size()
    Pd = G.sta_get_paths()
    n2 = G.extract_critical_paths(-1, cfg.K, False)
    tot2 = G.sta_get_paths_size()
    Pd2 = G.sta_get_paths()
    same = all(torch.equal(Pd[k], Pd2[k]) for k in Pd)
    del Pd2
    P = {k: v.cpu().numpy() for k, v in Pd.items()}
    del Pd
    n_pairs = G.attraction_update_pairs(10.0, 0.2)
    return dict(nl=nl, T=T, tm=tm, G=G, x=x, y=y, wns=wns, tns=tns, K=cfg.K, n1=n1, n2=n2, tot1=tot1,
                tot2=tot2, same=same, n_pairs=n_pairs, P=P)


def _failing_endpoints(nl, tm):
    ct = nl.cell_type[nl.pin_cell]
    ep = np.nonzero((nl.pin_dir == 0) & ((ct == netgen.FF) | (ct == netgen.PO)))[0]
    return ep[tm["slack"][ep] < 0.0]


def test_sta_every_pin(run):
    check_sta(run["G"], run["tm"], run["T"], TOL32)
    assert run["tns"] == pytest.approx(run["tm"]["tns"], rel=1e-6)
    assert run["wns"] == pytest.approx(run["tm"]["wns"], rel=1e-6)


def test_all_endpoint_extraction_totals(run):
    nl, tm, K = run["nl"], run["tm"], run["K"]
    n_viol, n_paths, n_pins = run["tot1"]
    ref_viol = _failing_endpoints(nl, tm)
    assert abs(n_viol - len(ref_viol)) <= 2, (n_viol, len(ref_viol))
    assert n_viol <= n_paths <= K * n_viol
    assert n_pins > 2 * n_paths
    assert run["n1"] == n_paths
    assert (run["n2"], run["tot2"]) == (run["n1"], run["tot1"])
    assert run["same"]  # the second extraction wrote the same bits
    assert run["n_pairs"] > 0


def test_paths_on_every_failing_endpoint(run):
    P, nl, tm = run["P"], run["nl"], run["tm"]
    d = compare_paths(nl, tm, run["T"], run["K"], False, P, TOL32, extra=1, detail=True)
    # every decided endpoint matched exactly inside compare_paths; with K = 32
    # the 32nd and 33rd paths of an endpoint are more often closer than the
    # slack tolerance (1e-3 ps + 1e-6 x ~4 us here, ~4 ps), so a few percent
    # of the endpoints are ambiguous and pass the validity checks instead
    assert d["checked"] + d["ambiguous"] >= len(_failing_endpoints(nl, tm))
    assert d["ambiguous"] <= 0.1 * (d["checked"] + d["ambiguous"]), d["ambiguous"]
    assert d["paths"] == len(P["ep"])
    print(f"\nstress path sets: {d['checked']} decided endpoints identical, {d['ambiguous']} ambiguous "
          f"({len(d['differ'])} of them with another set), {d['paths']} paths, "
          f"max |slack - oracle| {d['max_slack_err']:.3g} ps")


def test_loss_and_gradient(run):
    nl, G, x, y = run["nl"], run["G"], run["x"], run["y"]
    rng = np.random.default_rng(9)
    sinks = np.nonzero(nl.pin_dir == 0)[0]
    pins = np.sort(rng.choice(sinks, len(sinks) // 4, replace=False)).astype(np.int32)
    w = rng.uniform(5.0, 20.0, len(pins)).astype(np.float32).astype(np.float64)
    G.attraction_set_pairs(pins, w)
    in_p = np.zeros(nl.n_pins, np.uint8)
    in_p[pins] = 1
    wf = np.zeros(nl.n_pins)
    wf[pins] = w
    beta = 2.5e-5
    pp, gx_r, gy_r = oracle.loss(nl, in_p, wf, beta)
    assert G.attraction_loss_fwd(x, y, beta).item() == pytest.approx(pp, rel=1e-6)
    gx, gy = G.attraction_loss_bwd(x, y, beta)
    g = np.concatenate([gx.cpu().numpy(), gy.cpu().numpy()]).astype(np.float64)
    gr = np.concatenate([gx_r, gy_r])
    assert np.linalg.norm(g - gr) / np.linalg.norm(gr) <= 1e-5
