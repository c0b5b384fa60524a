"""Parity at the stress size: 3M movable cells (3.3M nets, ~10.5M pins), depth
120, clock at 0.8x the largest arrival, K = 32 paths per failing endpoint.

* STA on every pin and WNS / TNS against the FP64 oracle.
* The extraction of all failing endpoints with K = 32 (the call of a timing
  iteration) is checked by its totals against the oracle's failing endpoints,
  and repeated for determinism; its paths are too many to materialise here
  (~2.6M paths, ~600M pins), so
* the K = 32 path sets of the 400 most critical endpoints are extracted and
  compared with the oracle's pin sequences under the margin rule.
* The pair update runs on the full path set; the loss and its gradient are
  checked with a seeded pair set.
"""
import numpy as np
import pytest
import torch

import netgen
import oracle
from parity_util import TOL32, check_sta, compare_paths, gpu_paths

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
    n2 = G.extract_critical_paths(-1, cfg.K, False)
    tot2 = G.sta_get_paths_size()
    n_pairs = G.attraction_update_pairs(10.0, 0.2)
    G.extract_critical_paths(400, cfg.K, False)
    P = gpu_paths(G)
    return dict(nl=nl, T=T, tm=tm, G=G, x=x, y=y, wns=wns, tns=tns, K=cfg.K, n1=n1, n2=n2, tot1=tot1,
                tot2=tot2, n_pairs=n_pairs, P=P)


def test_sta_every_pin(run):
    check_sta(run["G"], run["tm"], run["T"], TOL32)
    assert run["tns"] == pytest.approx(run["tm"]["tns"], rel=1e-6)
    assert run["wns"] == pytest.approx(run["tm"]["wns"], rel=1e-6)


def test_all_endpoint_extraction_totals(run):
    nl, tm, K = run["nl"], run["tm"], run["K"]
    n_viol, n_paths, n_pins = run["tot1"]
    ref_viol = oracle.topk(nl, tm, -1, 1)["viol"]
    assert abs(n_viol - len(ref_viol)) <= 2, (n_viol, len(ref_viol))
    assert n_viol <= n_paths <= K * n_viol
    assert n_pins > 2 * n_paths
    assert run["n1"] == n_paths
    assert (run["n2"], run["tot2"]) == (run["n1"], run["tot1"])  # deterministic
    assert run["n_pairs"] > 0


def test_most_critical_endpoint_paths(run):
    P, nl, tm = run["P"], run["nl"], run["tm"]
    assert len(P["viol"]) >= 400 and len(np.unique(P["ep"])) == 400
    checked, amb = compare_paths(nl, tm, run["T"], run["K"], False, P, TOL32, endpoints=P["viol"][:400])
    # every endpoint whose set is decided by more than the slack tolerance
    # (1e-3 ps + 1e-6 x ~3.7 us here, ~3.7 ps) matches exactly; with K = 32
    # the 32nd and 33rd paths of a critical endpoint are often closer than
    # that, so a share of the endpoints is ambiguous by the margin rule
    assert checked >= 300, (checked, amb)


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
