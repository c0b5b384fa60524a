"""Parity of report_timing(n) (Section III-B, Table I) with the FP64 oracle,
through the C ABI.

The oracle follows the paper's definition (the n worst endpoints, the n worst
paths of each, the n worst of those); the CUDA path searches the prefix tree
of all paths under a shrinking slack bound.  Compared:
* the reported slacks, worst first, element by element;
* every reported pin sequence is a real start -> end path, and its slack
  recomputed in FP64 from the oracle's delays is the reported one;
* the path sets, except paths within the slack tolerance of the n-th slack
  (where either choice is correct) or, without keep_nonneg, of zero;
* determinism, the edge cases (n = 0, n beyond the number of paths, no
  failing endpoint, n < 0, calls out of order) and the pair update over the
  reported paths.
At 1.2M cells, where the oracle cannot take n^2 paths, properties that fix the
answer at any size are checked: the reported paths of an endpoint are its
lowest-slack ones (the oracle's top-k of that endpoint, on sampled
endpoints), no other path of such an endpoint lies below the n-th slack, and
no endpoint missing from the report has a slack below it.
"""
import numpy as np
import pytest
import torch

import netgen
import oracle
from parity_util import gpu_paths, paths_by_endpoint, tol_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2503_11674_b300.build import build
    build()


def _graph(nl, prec):
    from paper_2503_11674_b300 import TimingGraph
    return TimingGraph(nl, prec)


def _setup(cfg, seed, prec):
    nl = netgen.generate(cfg, seed)
    T = oracle.clock_period(nl, netgen.CONFIGS[cfg].t_factor)
    tm = oracle.sta(nl, T=T)
    G = _graph(nl, prec)
    x = torch.tensor(nl.x, dtype=G.dtype, device="cuda")
    y = torch.tensor(nl.y, dtype=G.dtype, device="cuda")
    return nl, T, tm, G, x, y


def _endpoints(nl):
    ct = nl.cell_type[nl.pin_cell]
    return np.nonzero((nl.pin_dir == 0) & ((ct == netgen.FF) | (ct == netgen.PO)))[0]


class _Checker:
    """FP64 slack of a pin sequence from the oracle's delays; asserts that the
    sequence is a start -> end path of the timing graph."""

    def __init__(self, nl, tm, T):
        self.nl, self.tm, self.T = nl, tm, T
        self.pin_net = np.repeat(np.arange(nl.n_nets), np.diff(nl.net_ptr))
        self.drv = nl.net_ptr[:-1]
        self.ct = nl.cell_type[nl.pin_cell]

    def slack(self, seq):
        nl, tm, pn, ct = self.nl, self.tm, self.pin_net, self.ct
        p0, e = seq[0], seq[-1]
        assert nl.pin_dir[p0] == 1 and ct[p0] in (netgen.FF, netgen.PI), seq
        assert nl.pin_dir[e] == 0 and ct[e] in (netgen.FF, netgen.PO), seq
        d = tm["dnet"][pn[p0]]
        for a, b in zip(seq[:-1], seq[1:]):
            if nl.pin_dir[b] == 0:   # net arc: from the net's driver
                assert self.drv[pn[b]] == a, (a, b)
                d += tm["tnet"][b]
            else:                    # cell arc: an input of the same combinational cell
                assert nl.pin_dir[a] == 0 and nl.pin_cell[a] == nl.pin_cell[b] and ct[b] == netgen.COMB, (a, b)
                d += tm["dnet"][pn[b]]
        return self.T - d


def _seqs(P):
    ptr, pins = P["pin_ptr"], P["pins"]
    return [tuple(pins[ptr[k]:ptr[k + 1]].tolist()) for k in range(len(P["ep"]))]


def _compare(nl, tm, T, tol, P, R, n, keep_nonneg):
    """GPU report P against the oracle's report R of the same n; returns the
    number of paths whose membership was decided beyond the tolerance."""
    ng, nr = len(P["ep"]), len(R["ep"])
    worst = min(R["slack"].min() if nr else 0.0, P["slack"].min() if ng else 0.0)
    tolp = tol[0] + tol[1] * (T + abs(worst))
    gs, rs = P["slack"].astype(np.float64), R["slack"]
    assert ng <= n and nr <= n
    if ng != nr:   # only where fewer than n paths fail, by paths within the tolerance of zero
        assert not keep_nonneg and max(ng, nr) < n + 1
        tail = gs[nr:] if ng > nr else rs[ng:]
        assert (np.abs(tail) <= tolp).all(), tail
    m = min(ng, nr)
    assert (np.abs(gs[:m] - rs[:m]) <= 2 * tolp).all(), np.abs(gs[:m] - rs[:m]).max()
    assert (np.diff(gs) >= 0).all()                          # worst first
    chk = _Checker(nl, tm, T)
    gseq, rseq = _seqs(P), _seqs(R)
    assert len(set(gseq)) == ng                              # no path twice
    true_g = np.array([chk.slack(s) for s in gseq])
    assert (np.abs(true_g - gs) <= tolp).all()
    assert [s[-1] for s in gseq] == P["ep"].tolist()
    # membership: decided unless within the tolerance of the n-th slack (or of 0)
    theta = rs[-1] if nr == n else (0.0 if not keep_nonneg else np.inf)
    lim = theta - 2 * tolp
    if not keep_nonneg:
        lim = min(lim, -2 * tolp)
    sure_r = {s for s, v in zip(rseq, rs) if v < lim}
    sure_g = {s for s, v in zip(gseq, true_g) if v < lim}
    gset, rset = set(gseq), set(rseq)
    assert sure_r <= gset, len(sure_r - gset)
    assert sure_g <= rset, len(sure_g - rset)
    # order: where the oracle's neighbouring slacks are separated beyond the
    # tolerance, the same path at the same rank (equal slacks may come in
    # another order: the GPU orders them by its expansion, not by R5)
    for i in range(m):
        sep_prev = i == 0 or rs[i] - rs[i - 1] > 4 * tolp
        sep_next = i == m - 1 or rs[i + 1] - rs[i] > 4 * tolp
        if sep_prev and sep_next and rs[i] < lim:
            assert gseq[i] == rseq[i], i
    return len(sure_r)


CASES = [("tiny", 1), ("tiny", 2), ("diff", 1)]


@pytest.mark.parametrize("keep_nonneg", [False, True])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("cfg,seed", CASES)
def test_report_timing_parity(cfg, seed, prec, keep_nonneg):
    nl, T, tm, G, x, y = _setup(cfg, seed, prec)
    tol = tol_of(G.dtype)
    G.sta_propagate(x, y, T)
    n_viol = int((tm["slack"][_endpoints(nl)] < 0).sum())
    ns = [1, 2, 37, 300]
    if cfg == "tiny":
        ns += [n_viol, 4 * n_viol]
    for n in ns:
        n_got = G.report_timing(n, keep_nonneg)
        P = gpu_paths(G)
        assert n_got == len(P["ep"]) == G.sta_get_paths_size()[1]
        R = oracle.report_timing(nl, tm, n, keep_nonneg)
        decided = _compare(nl, tm, T, tol, P, R, n, keep_nonneg)
        # all but a few paths near the boundary are decided beyond the tolerance
        assert decided >= 0.8 * (len(R["ep"]) - 1) - 1, (n, decided, len(R["ep"]))


def test_report_timing_is_deterministic_and_switches_modes():
    nl, T, tm, G, x, y = _setup("diff", 2, "fp32")
    G.sta_propagate(x, y, T)
    G.report_timing(500)
    a = gpu_paths(G)
    G.report_timing(500)
    b = gpu_paths(G)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])
    # report_timing_endpoint after report_timing, and back
    G.extract_critical_paths(-1, 4, False)
    c = gpu_paths(G)
    assert len(c["ep"]) >= len(c["viol"])
    G.report_timing(500)
    d = gpu_paths(G)
    for k in a:
        np.testing.assert_array_equal(a[k], d[k])


def test_report_timing_edge_cases():
    from paper_2503_11674_b300._abi import TdpError, STATUS_NAMES
    nl, T, tm, G, x, y = _setup("tiny", 3, "fp32")
    with pytest.raises(TdpError) as ei:   # before sta_propagate
        G.report_timing(5)
    assert STATUS_NAMES[ei.value.status] == "TDP_ERR_STATE"
    G.sta_propagate(x, y, T)
    with pytest.raises(TdpError) as ei:
        G.report_timing(-1)
    assert STATUS_NAMES[ei.value.status] == "TDP_ERR_INVALID"
    assert G.report_timing(0) == 0
    assert G.sta_get_paths_size()[1:] == (0, 0)
    # nothing fails at 10 T: no path, unless non-negative ones are kept
    G.sta_propagate(x, y, 10 * T)
    assert G.report_timing(50) == 0
    P = gpu_paths(G)
    assert len(P["viol"]) == 0 and len(P["ep"]) == 0
    assert G.report_timing(50, keep_nonneg=True) == 50
    tm10 = oracle.sta(nl, T=10 * T)
    _compare(nl, tm10, 10 * T, tol_of(G.dtype), gpu_paths(G), oracle.report_timing(nl, tm10, 50, True), 50, True)


def test_report_timing_more_than_all_paths():
    """A hand-built design with 11 paths in all: n = 100 reports all of them."""
    cells, nets = [], []
    for i in range(8):
        L = 100.0 * (i + 1)
        b = len(cells)
        cells += [{"type": "PI", "x": 0.0, "y": 50.0 * i, "rdrv": 1.0},
                  {"type": "COMB", "x": L, "y": 50.0 * i, "rdrv": 1.0},
                  {"type": "PO", "x": 2 * L, "y": 50.0 * i}]
        nets += [[(b, 0.0), (b + 1, 1.0)], [(b + 1, 0.0), (b + 2, 1.0)]]
    b = len(cells)
    cells += [{"type": "PI", "x": 0.0, "y": -50.0 * k - 50.0, "rdrv": 1.0} for k in range(3)]
    cells += [{"type": "COMB", "x": 10.0, "y": -100.0, "rdrv": 1.0}, {"type": "PO", "x": 20.0, "y": -100.0}]
    nets += [[(b + k, 0.0), (b + 3, 1.0)] for k in range(3)]
    nets += [[(b + 3, 0.0), (b + 4, 1.0)]]
    nl = netgen.from_lists(cells, nets)
    for prec in ("fp32", "fp64"):
        G = _graph(nl, prec)
        x = torch.tensor(nl.x, dtype=G.dtype, device="cuda")
        y = torch.tensor(nl.y, dtype=G.dtype, device="cuda")
        G.sta_propagate(x, y, 0.0)
        tm = oracle.sta(nl, T=0.0)
        for n in (1, 5, 11, 100):
            assert G.report_timing(n) == min(n, 11)
            _compare(nl, tm, 0.0, tol_of(G.dtype), gpu_paths(G), oracle.report_timing(nl, tm, n), n, False)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_pair_update_over_reported_paths(prec):
    """Eq. (w_ij) over the paths of report_timing(n): the oracle's update of
    the same path set (the GPU's paths and slacks, the GPU's WNS)."""
    nl, T, tm, G, x, y = _setup("diff", 1, prec)
    wns, _ = G.sta_propagate(x, y, T)
    w0, w1 = 10.0, 0.2
    G.report_timing(2000)
    P = gpu_paths(G)
    n_pairs = G.attraction_update_pairs(w0, w1)
    pins, w = G.attraction_get_pairs()
    pins, w = pins.cpu().numpy(), w.cpu().numpy().astype(np.float64)
    in_p, w_ref = oracle.update_pairs(nl, {"slack": P["slack"].astype(np.float64), "pin_ptr": P["pin_ptr"],
                                           "pins": P["pins"]}, wns, w0, w1)
    assert n_pairs == len(pins) == int(in_p.sum())
    np.testing.assert_array_equal(np.sort(pins), np.nonzero(in_p)[0])
    occ = np.zeros(nl.n_pins)
    for k in range(len(P["ep"])):
        occ[P["pins"][P["pin_ptr"][k]:P["pin_ptr"][k + 1]][1::2]] += 1
    wg = np.zeros(nl.n_pins)
    wg[pins] = w
    wtol = occ * w1 * 2.0 ** -22 + 2.0 ** -22 * np.abs(w_ref) + 1e-9
    assert (np.abs(wg - w_ref) <= wtol).all(), np.abs(wg - w_ref).max()


# ------------------------------------------------------------ full size ----

@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    nl, T, tm, G, x, y = _setup("1.2M", 1, "fp32")
    G.sta_propagate(x, y, T)
    eps = _endpoints(nl)
    n_viol = int((tm["slack"][eps] < 0).sum())
    return nl, T, tm, G, eps, n_viol


@pytest.mark.parametrize("mult", [1, 10])
def test_report_timing_full_size(big, mult):
    """report_timing(n) at 1.2M cells with n = the failing endpoints (20k) and
    10x that, the two settings of Table I."""
    nl, T, tm, G, eps, n_viol = big
    n = mult * n_viol
    tol = tol_of(G.dtype)
    assert G.report_timing(n) == n
    P = gpu_paths(G)
    gs = P["slack"].astype(np.float64)
    tolp = tol[0] + tol[1] * (T + abs(gs[0]))
    assert (np.diff(gs) >= 0).all()
    theta = gs[-1]
    chk = _Checker(nl, tm, T)
    ptr, pins = P["pin_ptr"], P["pins"]
    rng = np.random.default_rng(5)
    for k in np.concatenate([[0, n - 1], rng.choice(n, 2000, replace=False)]):
        seq = pins[ptr[k]:ptr[k + 1]].tolist()
        assert seq[-1] == P["ep"][k]
        assert abs(chk.slack(seq) - gs[k]) <= tolp
    # no endpoint outside the report has a slack below the n-th
    rep = np.unique(P["ep"])
    out = np.setdiff1d(eps, rep)
    assert (tm["slack"][out] >= theta - 2 * tolp).all()
    # per endpoint: its reported paths are its lowest-slack ones, and its next
    # path is not below the n-th slack
    cnt = {int(e): c for e, c in zip(*np.unique(P["ep"], return_counts=True))}
    small = [e for e, c in cnt.items() if c <= 1500]
    pick = list(rng.choice(small, min(12, len(small)), replace=False))
    worst_ep = int(P["ep"][0])
    if cnt[worst_ep] <= 4000:
        pick.append(worst_ep)
    for e in pick:
        e = int(e)
        m = cnt[e]
        ref = paths_by_endpoint(oracle.topk(nl, tm, -1, m + 1, True, endpoints=[e]))[e]
        mine = [(float(gs[k]), tuple(pins[ptr[k]:ptr[k + 1]].tolist())) for k in np.nonzero(P["ep"] == e)[0]]
        assert len(mine) == m
        np.testing.assert_allclose([p[0] for p in mine], [p[0] for p in ref[:m]], atol=2 * tolp, rtol=0)
        if len(ref) > m:
            assert ref[m][0] >= theta - 2 * tolp
        lim = theta - 2 * tolp
        assert {p[1] for p in ref[:m] if p[0] < lim} <= {p[1] for p in mine}
