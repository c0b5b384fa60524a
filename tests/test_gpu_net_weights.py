"""net_weights_update (the net-weighting baseline: weights from the worst
pin slack on each net, with momentum) against the FP64 oracle, through the
C ABI, over three updates at three placements.

Tolerance, derived from the slack tolerance of the STA: a net's criticality
c = min(1, max(0, -s) / |WNS|) moves by at most (tol_s + tol_WNS) / |WNS|
when its slack s moves by tol_s and the WNS by tol_WNS (max(0, .) and min(1, .)
are 1-Lipschitz, and |s| <= |WNS| where c < 1); the momentum update
w <- alpha w + (1 - alpha)(1 + gamma c) carries an error e to alpha e +
(1 - alpha) gamma dc, so after any number of updates the weights differ by
at most gamma max dc, plus a few rounding units of the weight per update.
The count of nets with negative slack may differ only by nets whose slack is
within tol_s of zero.
"""
import numpy as np
import pytest
import torch

import netgen
import oracle
from parity_util import check_net_weights, tol_of

pytestmark = pytest.mark.gpu

ALPHA, GAMMA = 0.5, 4.0


def _graph(nl, prec):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2503_11674_b300 import TimingGraph
    from paper_2503_11674_b300.build import build
    build()
    return TimingGraph(nl, prec)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("cfg,seed", [("tiny", 1), ("diff", 1), ("mid", 1)])
def test_net_weights_parity_over_three_updates(cfg, seed, prec):
    nl = netgen.generate(cfg, seed)
    T = oracle.clock_period(nl, netgen.CONFIGS[cfg].t_factor)
    G = _graph(nl, prec)
    tol = tol_of(G.dtype)
    assert (G.net_weights_get().cpu().numpy() == 1.0).all()   # every weight starts at 1
    rng = np.random.default_rng(seed)
    x, y = nl.x.copy(), nl.y.copy()
    w_ref = None
    for k in range(1, 4):
        xg = torch.tensor(x, dtype=G.dtype, device="cuda")
        yg = torch.tensor(y, dtype=G.dtype, device="cuda")
        G.sta_propagate(xg, yg, T)
        n_gpu = G.net_weights_update(ALPHA, GAMMA)
        # the oracle on the same (rounded) positions
        tm = oracle.sta(nl, xg.double().cpu().numpy(), yg.double().cpu().numpy(), T)
        w_ref, n_ref = oracle.net_weights(nl, tm, ALPHA, GAMMA, w_ref)
        w_gpu = G.net_weights_get().double().cpu().numpy()
        eps = 2.0 ** -23 if G.dtype == torch.float32 else 2.0 ** -52
        check_net_weights(nl, tm, T, w_gpu, w_ref, n_gpu, n_ref, tol, eps, k, GAMMA)
        assert n_gpu > 0 and (w_gpu >= 1.0 - 1e-6).all() and (w_gpu <= 1.0 + GAMMA + 1e-5).all()
        x, y = netgen.perturb(x, y, nl.cell_fixed, 20.0, rng)
    G.close()


def test_net_weights_stream_order_reset_and_errors():
    from paper_2503_11674_b300._abi import TDP_ERR_INVALID, TDP_ERR_STATE, TdpError
    nl = netgen.generate("tiny", 2)
    T = oracle.clock_period(nl, 0.9)
    G = _graph(nl, "fp32")
    x = torch.tensor(nl.x, dtype=torch.float32, device="cuda")
    y = torch.tensor(nl.y, dtype=torch.float32, device="cuda")
    with pytest.raises(TdpError) as ei:
        G.net_weights_update(ALPHA, GAMMA)
    assert ei.value.status == TDP_ERR_STATE
    G.sta_propagate(x, y, T)
    for a, g in ((-0.1, 1.0), (1.5, 1.0), (0.5, -1.0), (0.5, float("inf")), (float("nan"), 1.0)):
        with pytest.raises(TdpError) as ei:
            G.net_weights_update(a, g)
        assert ei.value.status == TDP_ERR_INVALID
    # stream-ordered calls (no host sync) give the same weights as synchronous ones
    G.net_weights_update(ALPHA, GAMMA, sync=False)
    G.net_weights_update(ALPHA, GAMMA, sync=False)
    w_async = G.net_weights_get().cpu().numpy()
    G.net_weights_reset()
    assert (G.net_weights_get().cpu().numpy() == 1.0).all()
    G.net_weights_update(ALPHA, GAMMA)
    G.net_weights_update(ALPHA, GAMMA)
    np.testing.assert_array_equal(G.net_weights_get().cpu().numpy(), w_async)
    # alpha = 1 holds the weights; alpha = 0 gives the target 1 + gamma c
    G.net_weights_update(1.0, GAMMA)
    np.testing.assert_array_equal(G.net_weights_get().cpu().numpy(), w_async)
    G.net_weights_update(0.0, 0.0)
    assert (G.net_weights_get().cpu().numpy() == 1.0).all()
    G.close()
