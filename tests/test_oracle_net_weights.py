"""Pins of the oracle's net weighting (the baseline of Section II-C and the
"w/o Path Extraction" ablation of Section IV), read as
    s_e = worst pin slack of net e,
    c_e = min(1, max(0, -s_e) / |WNS|)   (0 when WNS = 0),
    w_e <- alpha w_e + (1 - alpha)(1 + gamma c_e),  w starting at 1.

* the three-pin net of Section III-A (driver A, sinks B and C, C at -500 ps,
  the path through B with positive slack) by hand, over three updates;
* the closed form of the momentum recurrence, w_k = t + alpha^k (w_0 - t),
  for a constant target t;
* monotonicity in the worst slack, the bounds 1 <= target <= 1 + gamma, and
  the cases WNS = 0 and non-negative slack;
* on synthetic netlists: the net's worst pin slack is its driver's slack
  (every sink's slack is at least its driver's), checked against the FP64
  STA pin by pin, so the reading needs nothing beyond STA.
"""
import numpy as np
import pytest

import netgen
import oracle


class _NL:
    def __init__(self, net_ptr):
        self.net_ptr = np.asarray(net_ptr, np.int32)
        self.n_nets = len(net_ptr) - 1


def _timing(slack, wns):
    return {"slack": np.asarray(slack, float), "wns": float(wns)}


def test_three_pin_net_by_hand():
    # net 0: driver A (pin 0) with sinks B (pin 1) and C (pin 2); C is on the
    # paths of slack -400 and -500, so its pin slack is -500, B's is +200; A,
    # the driver, carries the worst of its sinks' slacks
    nl = _NL([0, 3])
    tm = _timing([-500.0, 200.0, -500.0], -500.0)
    alpha, gamma = 0.5, 4.0
    w, n = oracle.net_weights(nl, tm, alpha, gamma)
    assert n == 1
    assert w[0] == pytest.approx(0.5 * 1.0 + 0.5 * (1.0 + 4.0 * 1.0))  # 3.0
    w, _ = oracle.net_weights(nl, tm, alpha, gamma, w)
    assert w[0] == pytest.approx(4.0)
    w, _ = oracle.net_weights(nl, tm, alpha, gamma, w)
    assert w[0] == pytest.approx(4.5)
    # half as critical as the WNS: target 1 + gamma / 2
    w, _ = oracle.net_weights(nl, _timing([-250.0, 10.0, -250.0], -500.0), alpha, gamma)
    assert w[0] == pytest.approx(0.5 + 0.5 * 3.0)


def test_momentum_closed_form():
    rng = np.random.default_rng(3)
    m = 200
    net_ptr = np.arange(0, 2 * m + 1, 2)
    slack = np.repeat(rng.uniform(-900.0, 300.0, m), 2)
    wns = slack.min()
    alpha, gamma = 0.7, 6.0
    w0 = rng.uniform(0.5, 5.0, m)
    c = np.minimum(1.0, np.maximum(0.0, -slack[0::2]) / -wns)
    t = 1.0 + gamma * c
    w = w0.copy()
    for k in range(1, 9):
        w, n = oracle.net_weights(_NL(net_ptr), _timing(slack, wns), alpha, gamma, w)
        np.testing.assert_allclose(w, t + alpha ** k * (w0 - t), rtol=1e-12, atol=1e-12)
        assert n == int((slack[0::2] < 0).sum())


def test_monotone_bounded_and_degenerate_cases():
    m = 101
    net_ptr = np.arange(0, 2 * m + 1, 2)
    s = np.linspace(-1000.0, 1000.0, m)
    slack = np.repeat(s, 2)
    alpha, gamma = 0.0, 5.0                                  # alpha = 0: the target itself
    w, n = oracle.net_weights(_NL(net_ptr), _timing(slack, -1000.0), alpha, gamma)
    assert (np.diff(w) <= 0).all()                           # worse slack, larger weight
    assert (w >= 1.0).all() and (w <= 1.0 + gamma).all()
    assert w[0] == 1.0 + gamma and (w[s >= 0] == 1.0).all()
    assert n == int((s < 0).sum())
    w, _ = oracle.net_weights(_NL(net_ptr), _timing(slack, 0.0), alpha, gamma)
    assert (w == 1.0).all()                                  # WNS = 0: nothing critical
    # alpha = 1: the weights do not move
    w1 = np.full(m, 2.5)
    w, _ = oracle.net_weights(_NL(net_ptr), _timing(slack, -1000.0), 1.0, gamma, w1)
    assert (w == 2.5).all()


@pytest.mark.parametrize("cfg,seed", [("tiny", 1), ("diff", 2)])
def test_worst_pin_slack_of_a_net_is_its_drivers(cfg, seed):
    nl = netgen.generate(cfg, seed)
    T = oracle.clock_period(nl, netgen.CONFIGS[cfg].t_factor)
    tm = oracle.sta(nl, T=T)
    npt = np.asarray(nl.net_ptr)
    worst = np.minimum.reduceat(tm["slack"], npt[:-1])
    drv = tm["slack"][npt[:-1]]
    np.testing.assert_allclose(worst, drv, rtol=0, atol=1e-9 * T)
    # the weights are those of the driver slacks
    alpha, gamma = 0.5, 4.0
    w, n = oracle.net_weights(nl, tm, alpha, gamma)
    c = np.minimum(1.0, np.maximum(0.0, -drv) / -tm["wns"])
    np.testing.assert_allclose(w, alpha + (1 - alpha) * (1 + gamma * c), rtol=1e-9, atol=1e-9)
    assert n == int((worst < 0).sum()) and n > 0
