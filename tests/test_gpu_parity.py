"""Parity of the CUDA library (through the C ABI) with the FP64 oracle."""
import numpy as np
import pytest
import torch

import netgen
import oracle
from golden_util import GOLDEN_NAMES, load
from parity_util import (TOL32, TOL64, check_sta, close, compare_paths, gpu_paths, paths_by_endpoint,
                         sta_scales, tol_of)

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


def _pos(nl, dtype, x=None, y=None):
    x = nl.x if x is None else x
    y = nl.y if y is None else y
    return (torch.tensor(np.asarray(x), dtype=dtype, device="cuda"),
            torch.tensor(np.asarray(y), dtype=dtype, device="cuda"))


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


# ------------------------------------------------------------ golden -------

@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("name", GOLDEN_NAMES)
def test_golden_circuits(name, prec):
    gj, nl = load(name)
    e = gj["expect"]
    G = _graph(nl, prec)
    x, y = _pos(nl, G.dtype)
    tol = 1e-4 if prec == "fp32" else 1e-9
    wns, tns = G.sta_propagate(x, y, gj["T"])
    assert wns == pytest.approx(e["wns"], abs=tol) and tns == pytest.approx(e["tns"], abs=tol)
    arr, req, slack = (_np(t) for t in G.sta_get_timing())
    tnet, cload, dnet = (_np(t) for t in G.sta_get_net_delays())
    for key, got in (("arr", arr), ("req", req), ("slack", slack), ("tnet", tnet), ("dnet", dnet),
                     ("cload", cload)):
        if key in e:
            np.testing.assert_allclose(got, e[key], atol=tol, rtol=0)
    n = G.extract_critical_paths(-1, gj["K"], False)
    P = gpu_paths(G)
    assert n == len(e["paths"])
    for k, ex in enumerate(e["paths"]):
        assert P["ep"][k] == ex["ep"]
        assert P["pins"][P["pin_ptr"][k]:P["pin_ptr"][k + 1]].tolist() == ex["pins"]
        assert P["slack"][k] == pytest.approx(ex["slack"], abs=tol)
    if "paths_keep_nonneg" in e:
        G.extract_critical_paths(-1, gj["K"], True)
        Q = gpu_paths(G)
        assert [Q["pins"][Q["pin_ptr"][k]:Q["pin_ptr"][k + 1]].tolist() for k in range(len(Q["ep"]))] == \
            [ex["pins"] for ex in e["paths_keep_nonneg"]]
        G.extract_critical_paths(-1, gj["K"], False)
    npairs = G.attraction_update_pairs(gj["w0"], gj["w1"])
    exp = {int(k): v for k, v in e["pairs_after_one_update"].items()}
    pins, w = G.attraction_get_pairs()
    assert npairs == len(exp)
    assert pins.cpu().tolist() == sorted(exp)
    np.testing.assert_allclose(_np(w), [exp[p] for p in sorted(exp)], rtol=1e-6, atol=1e-6)
    loss = G.attraction_loss_fwd(x, y, gj["beta"])
    assert loss.item() == pytest.approx(e["pp"], rel=1e-6)
    gx, gy = G.attraction_loss_bwd(x, y, gj["beta"])
    np.testing.assert_allclose(_np(gx), e["gx"], atol=1e-3 * max(1, np.abs(e["gx"]).max()) * 1e-3)
    np.testing.assert_allclose(_np(gy), e["gy"], atol=1e-3 * max(1, np.abs(e["gy"]).max()) * 1e-3)
    if "pairs_after_two_updates" in e:
        G.attraction_update_pairs(gj["w0"], gj["w1"])
        pins, w = G.attraction_get_pairs()
        exp2 = {int(k): v for k, v in e["pairs_after_two_updates"].items()}
        np.testing.assert_allclose(_np(w), [exp2[p] for p in pins.cpu().tolist()], rtol=1e-6)


# ------------------------------------------------------ random netlists ----

CASES = [("tiny", 1), ("tiny", 2), ("diff", 1), ("mid", 1)]


def _setup(cfg, seed, prec):
    nl = netgen.generate(cfg, seed)
    T = oracle.clock_period(nl, netgen.CONFIGS[cfg].t_factor)
    tm = oracle.sta(nl, T=T)
    G = _graph(nl, prec)
    x, y = _pos(nl, G.dtype)
    return nl, T, tm, G, x, y


def _endpoints(nl):
    ct = nl.cell_type[nl.pin_cell]
    return np.nonzero((nl.pin_dir == 0) & ((ct == netgen.FF) | (ct == netgen.PO)))[0]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("cfg,seed", CASES)
def test_sta_parity(cfg, seed, prec):
    nl, T, tm, G, x, y = _setup(cfg, seed, prec)
    tol = tol_of(G.dtype)
    wns, tns = G.sta_propagate(x, y, T)
    _, _, slack = check_sta(G, tm, T, tol)
    ep = _endpoints(nl)
    s_gpu = slack[ep]
    # the FP64 reduction of the GPU's own endpoint slacks
    neg = s_gpu[s_gpu < 0]
    assert tns == pytest.approx(neg.sum(), rel=1e-12, abs=1e-9)
    assert wns == (neg.min() if len(neg) else 0.0)
    if prec == "fp64":
        assert tns == pytest.approx(tm["tns"], rel=1e-9)
        assert wns == pytest.approx(tm["wns"], rel=1e-9)
    else:
        # end-to-end FP32 against the sum of the per-endpoint tolerances
        sc = sta_scales(tm, T)[2]
        ep_tol = TOL32[0] + TOL32[1] * sc[ep]
        assert abs(tns - tm["tns"]) <= ep_tol.sum()
        assert abs(wns - tm["wns"]) <= ep_tol.max()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("keep_nonneg", [False, True])
@pytest.mark.parametrize("cfg,seed", CASES)
def test_extract_parity(cfg, seed, prec, keep_nonneg):
    if keep_nonneg and cfg == "mid":
        pytest.skip("keep_nonneg covered on the smaller netlists")
    nl, T, tm, G, x, y = _setup(cfg, seed, prec)
    K = netgen.CONFIGS[cfg].K
    tol = tol_of(G.dtype)
    G.sta_propagate(x, y, T)
    n = G.extract_critical_paths(-1, K, keep_nonneg)
    P = gpu_paths(G)
    assert n == len(P["ep"])
    # failing endpoints, sorted by (slack, pin)
    ref = oracle.topk(nl, tm, -1, 1)
    tolp = tol[0] + tol[1] * T
    sure = np.abs(tm["slack"][ref["viol"]]) > tolp
    ep_all = _endpoints(nl)
    near0 = ep_all[np.abs(tm["slack"][ep_all]) <= tolp]
    assert set(ref["viol"][sure].tolist()) <= set(P["viol"].tolist()) <= \
        set(ref["viol"].tolist()) | set(near0.tolist())
    s_in_gpu_order = tm["slack"][P["viol"]]
    assert (np.diff(s_in_gpu_order) >= -2 * tolp).all()
    checked, amb = compare_paths(nl, tm, T, K, keep_nonneg, P, tol)
    assert checked > 0 and amb <= max(2, 0.05 * (checked + amb)), (checked, amb)
    # every path: consecutive pins are connected, and it ends at its endpoint
    ptr, pins = P["pin_ptr"], P["pins"]
    for k in range(min(len(P["ep"]), 2000)):
        seq = pins[ptr[k]:ptr[k + 1]]
        assert seq[-1] == P["ep"][k] and nl.pin_dir[seq[0]] == 1
        assert (nl.pin_dir[seq[0::2]] == 1).all() and (nl.pin_dir[seq[1::2]] == 0).all()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("cfg,seed", [("tiny", 1), ("diff", 1), ("mid", 1)])
def test_pair_update_parity(cfg, seed, prec):
    nl, T, tm, G, x, y = _setup(cfg, seed, prec)
    K = netgen.CONFIGS[cfg].K
    tol = tol_of(G.dtype)
    w0, w1 = 10.0, 0.2
    G.sta_propagate(x, y, T)
    G.extract_critical_paths(-1, K, False)
    Pg = gpu_paths(G)
    n_pairs = G.attraction_update_pairs(w0, w1)
    pins, w = G.attraction_get_pairs()
    pins, w = pins.cpu().numpy(), _np(w)
    assert n_pairs == len(pins)
    Pr = oracle.topk(nl, tm, -1, K)
    in_p, w_ref = oracle.update_pairs(nl, Pr, tm["wns"], w0, w1)
    # exclude sinks touched by endpoints whose path set is not decided beyond tolerance
    tolp = tol[0] + tol[1] * T
    full = paths_by_endpoint(oracle.topk(nl, tm, -1, K + 1, True))
    bad = set()
    for e, lst in full.items():
        ex = [p for p in lst[:K] if p[0] < 0]
        nxt = lst[len(ex)] if len(lst) > len(ex) else None
        if abs(tm["slack"][e]) <= tolp or (nxt is not None and ex and nxt[0] - ex[-1][0] <= tolp) \
                or (ex and ex[-1][0] >= -tolp) or (nxt is not None and len(ex) < K and nxt[0] <= tolp):
            bad.add(e)
    touched_bad = set()
    for src in (paths_by_endpoint(Pr), paths_by_endpoint(Pg)):
        for e, lst in src.items():
            if e in bad:
                for _, seq in lst:
                    touched_bad.update(seq[1::2])
    ok = np.ones(nl.n_pins, bool)
    ok[list(touched_bad)] = False
    mine = np.zeros(nl.n_pins, bool)
    mine[pins] = True
    np.testing.assert_array_equal(mine[ok], in_p.astype(bool)[ok])
    wg = np.zeros(nl.n_pins)
    wg[pins] = w
    # occurrences per sink bound the accumulated error of slack / WNS
    occ = np.zeros(nl.n_pins)
    for k in range(len(Pr["ep"])):
        occ[Pr["pins"][Pr["pin_ptr"][k]:Pr["pin_ptr"][k + 1]][1::2]] += 1
    wtol = occ * w1 * (2 * tolp / abs(tm["wns"]) + 2.0 ** -23) + 1e-6 * np.abs(w_ref) + 1e-9
    sel = ok & (in_p > 0)
    assert (np.abs(wg[sel] - w_ref[sel]) <= wtol[sel]).all(), np.abs(wg[sel] - w_ref[sel]).max()
    assert sel.sum() > 0.9 * in_p.sum()


def _random_pairs(nl, seed, frac=0.4):
    rng = np.random.default_rng(seed)
    sinks = np.nonzero(nl.pin_dir == 0)[0]
    pins = np.sort(rng.choice(sinks, int(frac * len(sinks)), replace=False)).astype(np.int32)
    w = rng.uniform(5.0, 20.0, len(pins))
    in_p = np.zeros(nl.n_pins, np.uint8)
    in_p[pins] = 1
    wfull = np.zeros(nl.n_pins)
    wfull[pins] = w
    return pins, w, in_p, wfull


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("cfg,seed", CASES)
def test_loss_parity(cfg, seed, prec):
    nl = netgen.generate(cfg, seed)
    G = _graph(nl, prec)
    x, y = _pos(nl, G.dtype)
    pins, w, in_p, wfull = _random_pairs(nl, seed)
    if prec == "fp32":
        w = w.astype(np.float32).astype(np.float64)   # the oracle sees the stored weights
        wfull[pins] = w
    G.attraction_set_pairs(pins, w)
    beta = 2.5e-5
    pp, gx_r, gy_r = oracle.loss(nl, in_p, wfull, beta, x=_np(x), y=_np(y))
    loss = G.attraction_loss_fwd(x, y, beta).item()
    gx, gy = (_np(t) for t in G.attraction_loss_bwd(x, y, beta))
    rl = 1e-6 if prec == "fp32" else 1e-12
    assert loss == pytest.approx(pp, rel=rl)
    g = np.concatenate([gx, gy])
    gr = np.concatenate([gx_r, gy_r])
    rel_l2 = np.linalg.norm(g - gr) / np.linalg.norm(gr)
    assert rel_l2 <= (1e-5 if prec == "fp32" else 1e-12), rel_l2


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("kind", ["quadratic", "hpwl", "euclid"])
def test_fused_loss_call_matches_separate_calls(kind, prec):
    """attraction_loss_fwd_bwd gives the loss and gradient of
    attraction_loss_fwd + attraction_loss_bwd bit for bit, with and without
    a gradient scale, after a pair update from extracted paths."""
    nl = netgen.generate("diff", 3)
    T = oracle.clock_period(nl, 0.9)
    G = _graph(nl, prec)
    x, y = _pos(nl, G.dtype)
    G.sta_propagate(x, y, T)
    G.extract_critical_paths(-1, 8, False)
    assert G.attraction_update_pairs(10.0, 0.2) > 0
    G.attraction_set_loss_kind(kind)
    beta = 2.5e-5
    for scale in (None, torch.tensor(0.75, dtype=torch.float64, device="cuda")):
        loss = G.attraction_loss_fwd(x, y, beta).item()
        gx, gy = (t.clone() for t in G.attraction_loss_bwd(x, y, beta, grad_scale=scale))
        l2, gx2, gy2 = G.attraction_loss_fwd_bwd(x, y, beta, grad_scale=scale)
        assert l2.item() == loss
        assert torch.equal(gx2, gx) and torch.equal(gy2, gy)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("kind", ["hpwl", "euclid", "quadratic"])
def test_loss_kind_parity(kind, prec):
    """HPWL and linear Euclidean pair distances (the ablation's losses) against
    the oracle; gradients compared away from pairs whose |dx|, |dy| or
    distance is within 1e-3 um of the kink (where FP32 rounding can flip a
    sign)."""
    nl = netgen.generate("diff", 7)
    G = _graph(nl, prec)
    x, y = _pos(nl, G.dtype)
    pins, w, in_p, wfull = _random_pairs(nl, 7)
    if prec == "fp32":
        w = w.astype(np.float32).astype(np.float64)
        wfull[pins] = w
    G.attraction_set_pairs(pins, w)
    G.attraction_set_loss_kind(kind)
    beta = 2.5e-5
    xr, yr = _np(x), _np(y)
    pp, gx_r, gy_r = oracle.loss(nl, in_p, wfull, beta, x=xr, y=yr, kind=kind)
    loss = G.attraction_loss_fwd(x, y, beta).item()
    gx, gy = (_np(t) for t in G.attraction_loss_bwd(x, y, beta))
    assert loss == pytest.approx(pp, rel=1e-6 if prec == "fp32" else 1e-12)
    pc, nptr = nl.pin_cell, nl.net_ptr
    px = xr[pc] + nl.pin_dx.astype(np.float64)
    py = yr[pc] + nl.pin_dy.astype(np.float64)
    near = np.zeros(nl.n_cells, bool)
    drv = np.repeat(nptr[:-1], np.diff(nptr))
    dx, dy = px - px[drv], py - py[drv]
    bad = (in_p > 0) & ((np.abs(dx) < 1e-3) | (np.abs(dy) < 1e-3) | (np.hypot(dx, dy) < 1e-3))
    near[pc[bad]] = True
    near[pc[drv[bad]]] = True
    ok = ~near
    g = np.concatenate([gx[ok], gy[ok]])
    gr = np.concatenate([gx_r[ok], gy_r[ok]])
    rel_l2 = np.linalg.norm(g - gr) / np.linalg.norm(gr)
    assert rel_l2 <= (1e-5 if prec == "fp32" else 1e-12), rel_l2
    G.attraction_set_loss_kind("quadratic")
    assert G.attraction_loss_fwd(x, y, beta).item() == pytest.approx(
        oracle.loss(nl, in_p, wfull, beta, x=xr, y=yr)[0], rel=1e-6 if prec == "fp32" else 1e-12)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_autograd_finite_differences(prec):
    """attraction_loss_bwd behind torch.autograd vs central differences, 1,000 cells."""
    from paper_2503_11674_b300 import attraction_loss
    nl = netgen.generate("diff", 1)
    G = _graph(nl, prec)
    pins, w, in_p, wfull = _random_pairs(nl, 3)
    if prec == "fp32":
        w = w.astype(np.float32).astype(np.float64)
        wfull[pins] = w
    G.attraction_set_pairs(pins, w)
    beta = 2.5e-5
    x, y = _pos(nl, G.dtype)
    x.requires_grad_(True)
    y.requires_grad_(True)
    loss = attraction_loss(G, x, y, beta)
    (3.0 * loss).backward()
    gx, gy = _np(x.grad) / 3.0, _np(y.grad) / 3.0
    pp, gx_r, gy_r = oracle.loss(nl, in_p, wfull, beta, x=_np(x), y=_np(y))
    g, gr = np.concatenate([gx, gy]), np.concatenate([gx_r, gy_r])
    assert np.linalg.norm(g - gr) / np.linalg.norm(gr) <= 1e-5
    rng = np.random.default_rng(7)
    movable = np.nonzero(nl.cell_fixed == 0)[0]
    cells = rng.choice(movable, 1000, replace=False)
    # Rounding bound of the FD numerator per cell.  A term beta w Q with
    # Q = dx^2 + dy^2 is evaluated from coordinates below 1,000 um, so dx and dy
    # carry an absolute error of about 4 eps 1000 and Q a relative error 4 eps;
    # both evaluations (+h, -h) contribute.  The FD quotient is the exact
    # derivative at the midpoint of the two perturbed positions, which differs
    # from the gradient at the cell by 2 beta (sum of its pair weights) times
    # the midpoint offset.
    eps = 2.0 ** -52 if prec == "fp64" else 2.0 ** -24
    pin_net = np.repeat(np.arange(nl.n_nets), np.diff(nl.net_ptr))
    drv = nl.net_ptr[:-1][pin_net]
    px = nl.x.astype(float)[nl.pin_cell] + nl.pin_dx
    py = nl.y.astype(float)[nl.pin_cell] + nl.pin_dy
    ddx, ddy = np.abs(px - px[drv]), np.abs(py - py[drv])
    on = in_p > 0
    err = beta * wfull * (8 * eps * 1000.0 * (ddx + ddy) + 4 * eps * (ddx ** 2 + ddy ** 2)) * on
    per_cell = np.zeros(nl.n_cells)
    np.add.at(per_cell, nl.pin_cell, err)
    np.add.at(per_cell, nl.pin_cell[drv], err)
    wsum = np.zeros(nl.n_cells)
    np.add.at(wsum, nl.pin_cell, wfull * on)
    np.add.at(wsum, nl.pin_cell[drv], wfull * on)
    h = 1e-3
    with torch.no_grad():
        for c in cells:
            for arr_, gref in ((x, gx), (y, gy)):
                v0 = arr_[c].item()
                arr_[c] = v0 + h
                vp = arr_[c].item()
                lp = G.attraction_loss_fwd(x, y, beta).item()
                arr_[c] = v0 - h
                vm = arr_[c].item()
                lm = G.attraction_loss_fwd(x, y, beta).item()
                arr_[c] = v0
                fd = (lp - lm) / (vp - vm)     # exact for a quadratic, at the midpoint
                bound = (2 * per_cell[c] + 8 * 2.0 ** -52 * abs(lp)) / (vp - vm) + \
                    2 * beta * wsum[c] * abs((vp + vm) / 2 - v0) + 1e-9 * abs(gref[c])
                assert abs(fd - gref[c]) <= bound, (c, fd, gref[c], bound)


def _pipeline(nl, T, prec, K=16):
    G = _graph(nl, prec)
    x, y = _pos(nl, G.dtype)
    r = [G.sta_propagate(x, y, T)]
    G.extract_critical_paths(-1, K, False)
    P = gpu_paths(G)
    G.attraction_update_pairs(10.0, 0.2)
    pins, w = G.attraction_get_pairs()
    loss = G.attraction_loss_fwd(x, y, 2.5e-5)
    gx, gy = G.attraction_loss_bwd(x, y, 2.5e-5)
    return (r, P, pins.cpu().numpy(), w.cpu().numpy(), loss.item(), gx.cpu().numpy(),
            gy.cpu().numpy(), [t.cpu().numpy() for t in G.sta_get_timing()])


def _assert_same(a, b):
    assert a[0] == b[0] and a[4] == b[4]
    assert a[1].keys() == b[1].keys()
    for k in a[1]:
        np.testing.assert_array_equal(a[1][k], b[1][k])
    for i in (2, 3, 5, 6):
        np.testing.assert_array_equal(a[i], b[i])
    for u, v in zip(a[7], b[7]):
        np.testing.assert_array_equal(u, v)


def test_full_pipeline_is_deterministic():
    nl = netgen.generate("mid", 2)
    T = oracle.clock_period(nl, 0.85)
    _assert_same(_pipeline(nl, T, "fp32"), _pipeline(nl, T, "fp32"))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_level_launches_match_single_launch_sweeps(prec, monkeypatch):
    """The per-level CUDA-graph sweeps (used where a cooperative launch cannot
    be resident) do the same arithmetic in the same order as the single-launch
    sweeps: every output is bit-identical."""
    nl = netgen.generate("mid", 5)
    T = oracle.clock_period(nl, 0.85)
    one = _pipeline(nl, T, prec)
    monkeypatch.setenv("TDP_LEVEL_GRAPHS", "1")
    lv = _pipeline(nl, T, prec)
    _assert_same(one, lv)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_wide_cells(prec, monkeypatch):
    """Cells of more than four inputs (15% of them, 5 to 10 inputs) take the
    one-input-at-a-time path of the forward sweep: STA on every pin and the
    paths of every failing endpoint against the oracle, and the single-launch
    sweeps bit-identical to the per-level launches."""
    nl = netgen.random_dag(3000, 300, 20, 0.15, 4)
    assert (np.bincount(nl.pin_cell[nl.pin_dir == 0], minlength=nl.n_cells) > 4).sum() > 300
    T = oracle.clock_period(nl, 0.9)
    tm = oracle.sta(nl, T=T)
    G = _graph(nl, prec)
    x, y = _pos(nl, G.dtype)
    tol = tol_of(G.dtype)
    G.sta_propagate(x, y, T)
    check_sta(G, tm, T, tol)
    G.extract_critical_paths(-1, 8, False)
    checked, amb = compare_paths(nl, tm, T, 8, False, gpu_paths(G), tol)
    assert checked > 0 and amb <= max(2, 0.05 * (checked + amb)), (checked, amb)
    G.close()
    one = _pipeline(nl, T, prec, 8)
    monkeypatch.setenv("TDP_LEVEL_GRAPHS", "1")
    _assert_same(one, _pipeline(nl, T, prec, 8))


def _pipeline_async(nl, T, prec):
    """Two timing iterations queued without host synchronisation (the backward
    sweep overlaps extraction, the pair update and the loss), then every
    result read back."""
    G = _graph(nl, prec)
    out = []
    rng = np.random.default_rng(3)
    for it in range(2):
        x, y = _pos(nl, G.dtype, nl.x + (rng.normal(0, 2, nl.n_cells) if it else 0),
                    nl.y + (rng.normal(0, 2, nl.n_cells) if it else 0))
        G.sta_propagate(x, y, T, sync=False)
        G.extract_critical_paths(-1, 8, False, sync=False)
        G.attraction_update_pairs(10.0, 0.2, sync=False)
        loss = G.attraction_loss_fwd(x, y, 2.5e-5)
        gx, gy = G.attraction_loss_bwd(x, y, 2.5e-5)
        timing = [t.cpu().numpy() for t in G.sta_get_timing()]
        pins, w = G.attraction_get_pairs()
        P = gpu_paths(G)
        res = (pins.cpu().numpy(), w.cpu().numpy(), loss.item(), gx.cpu().numpy(), gy.cpu().numpy(), timing)
        out.append((G.sta_propagate(x, y, T), P) + res)
    return out


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_overlapped_backward_sweep_matches_serial(prec, monkeypatch):
    """The backward sweep on the library's second stream (beside extraction,
    pair update and loss) gives the same bits as the sweep in stream order."""
    nl = netgen.generate("mid", 6)
    T = oracle.clock_period(nl, 0.85)
    over = _pipeline_async(nl, T, prec)
    monkeypatch.setenv("TDP_SERIAL_BWD", "1")
    ser = _pipeline_async(nl, T, prec)
    for a, b in zip(over, ser):
        _assert_same(a, b)


@pytest.mark.parametrize("sms", ["1", "60", "-1"])
def test_backward_sweep_split_does_not_change_results(sms, monkeypatch):
    """The backward sweep started with net RC on its own SMs (one of them, 60
    of them, or after the forward sweep with TDP_BWD_SMS=-1) gives the bits of
    the default split: the SM split only moves work between the sweeps."""
    nl = netgen.generate("mid", 7)
    T = oracle.clock_period(nl, 0.85)
    ref = _pipeline_async(nl, T, "fp32")
    monkeypatch.setenv("TDP_BWD_SMS", sms)
    got = _pipeline_async(nl, T, "fp32")
    for a, b in zip(ref, got):
        _assert_same(a, b)


# --------------------------------------------------------- edge cases ------

def test_no_violation_and_empty_pairs():
    nl = netgen.generate("tiny", 4)
    G = _graph(nl, "fp32")
    x, y = _pos(nl, G.dtype)
    T = 10 * oracle.clock_period(nl, 1.0)
    assert G.sta_propagate(x, y, T) == (0.0, 0.0)
    assert G.extract_critical_paths(-1, 8, False) == 0
    assert G.sta_get_paths_size() == (0, 0, 0)
    assert G.attraction_update_pairs(10.0, 0.2) == 0
    assert G.attraction_loss_fwd(x, y, 1.0).item() == 0.0
    gx, gy = G.attraction_loss_bwd(x, y, 1.0)
    assert not gx.any() and not gy.any()
    # keep_nonneg still has no failing endpoint to search from
    assert G.extract_critical_paths(-1, 8, True) == 0


@pytest.mark.parametrize("K", [1, 2, 32])
def test_k_extremes_and_endpoint_limit(K):
    nl = netgen.generate("tiny", 2)
    T = oracle.clock_period(nl, 0.9)
    tm = oracle.sta(nl, T=T)
    G = _graph(nl, "fp64")
    x, y = _pos(nl, G.dtype)
    G.sta_propagate(x, y, T)
    G.extract_critical_paths(-1, K, False)
    P = gpu_paths(G)
    checked, amb = compare_paths(nl, tm, T, K, False, P, TOL64, endpoints=P["viol"])
    assert amb == 0 and checked == len(P["viol"])
    G.extract_critical_paths(5, K, False)
    Q = gpu_paths(G)
    assert set(Q["ep"].tolist()) == set(P["viol"][:5].tolist())
    sel = np.isin(P["ep"], P["viol"][:5])
    np.testing.assert_array_equal(Q["pins"], P["pins"][np.concatenate(
        [np.arange(P["pin_ptr"][k], P["pin_ptr"][k + 1]) for k in np.nonzero(sel)[0]])])


def test_out_of_order_calls_return_state_errors():
    from paper_2503_11674_b300 import _abi
    nl = netgen.generate("tiny", 1)
    G = _graph(nl, "fp32")
    with pytest.raises(_abi.TdpError) as ei:
        G.extract_critical_paths(-1, 4)
    assert ei.value.status == _abi.TDP_ERR_STATE
    with pytest.raises(_abi.TdpError) as ei:
        G.attraction_update_pairs()
    assert ei.value.status == _abi.TDP_ERR_STATE
    x, y = _pos(nl, G.dtype)
    G.sta_propagate(x, y, 1e3)
    with pytest.raises(_abi.TdpError) as ei:
        G.extract_critical_paths(-1, 33)
    assert ei.value.status == _abi.TDP_ERR_INVALID
    with pytest.raises(_abi.TdpError) as ei:
        G.attraction_set_pairs(np.array([0], np.int32), np.array([1.0]))  # pin 0 is a driver
    assert ei.value.status == _abi.TDP_ERR_INVALID



def test_grid_wait_gives_up_and_device_stays_usable():
    """The grid-wide wait of the single-launch sweeps is bounded: a barrier
    that can never complete records the timeout status and the kernel returns,
    leaving the context usable."""
    import ctypes as C
    from paper_2503_11674_b300 import _abi
    lib = _abi.load()
    gave_up = C.c_int32(-1)
    _abi.check("tdp_selftest_grid_wait", lib.tdp_selftest_grid_wait(2.0, C.addressof(gave_up)))
    assert gave_up.value == 1
    nl = netgen.generate("tiny", 3)
    T = oracle.clock_period(nl, 0.9)
    G = _graph(nl, "fp32")
    x, y = _pos(nl, G.dtype)
    G.sta_propagate(x, y, T)
    check_sta(G, oracle.sta(nl, nl.x, nl.y, T), T, TOL32)
