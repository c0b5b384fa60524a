"""Pin the FP64 oracle to things other than itself.

* Elmore delay (Eq. (8)): a generic RC-tree Elmore computation on a star net
  whose branches are discretised into pi-segment ladders, plus the driver
  resistance at the root, must give d - d0 + t_net for every sink.
* report_timing_endpoint (Section III-B): brute-force enumeration of every
  start -> end path on small random DAGs, sorted by slack and by the pin
  sequence read from the endpoint, must equal the oracle's top-K.
* STA invariants (Section II-B): translation invariance, WNS = min pin slack,
  TNS = sum of negative endpoint slacks, pin slack <= slack of every
  extracted path through it, rank-1 path slack = endpoint slack.
* Eq. (w_ij): the literal worst-first traversal equals the closed form
  w0 + (w1/WNS)(sum slack - min slack) for new pairs and
  w + (w1/WNS) sum slack for pairs already in P.
* Eq. (9) loss: central differences (exact for a quadratic up to rounding),
  sum of gradients = 0 (translation invariance), Euler's identity
  sum(x dPP/dx + y dPP/dy) = 2 PP (PP homogeneous of degree 2, zero offsets).
* HPWL and linear Euclidean pair distances (the ablation of Section IV): a
  hand-computed 3-4-5 pair, Euler's identity of degree 1, translation
  invariance and central differences away from the kinks.
"""
import itertools

import numpy as np
import pytest

import netgen
import oracle

SMALL = netgen.NetlistConfig("small", 36, 6, 44, 5, 0.5, 4, 0.0, 0.8, 6, offsets=True)


# ---------------------------------------------------------------- Elmore ----

def _elmore_tree(parent, R, Cnode):
    """Elmore delay of every node: sum over the root path of R_e * C_downstream."""
    n = len(parent)
    down = np.array(Cnode, dtype=float)
    for v in range(n - 1, 0, -1):          # nodes are numbered parent-before-child
        down[parent[v]] += down[v]
    delay = np.zeros(n)
    for v in range(1, n):
        delay[v] = delay[parent[v]] + R[v] * down[v]
    return delay


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_elmore_matches_rc_tree(seed):
    rng = np.random.default_rng(seed)
    fan = int(rng.integers(1, 6))
    cells = [{"type": "PI", "x": float(rng.uniform(0, 500)), "y": float(rng.uniform(0, 500)),
              "rdrv": float(rng.uniform(0.5, 2))}]
    for _ in range(fan):
        cells.append({"type": "PO", "x": float(rng.uniform(0, 500)), "y": float(rng.uniform(0, 500))})
    net = [(0, 1.0, float(rng.uniform(-1, 1)), float(rng.uniform(-1, 1)))]
    for k in range(fan):
        net.append((k + 1, float(rng.uniform(1, 3)), float(rng.uniform(-1, 1)), float(rng.uniform(-1, 1))))
    nl = netgen.from_lists(cells, [net])
    tm = oracle.sta(nl, T=0.0)

    # RC tree: node 0 = driver output (behind R_drv), node 1 = driver pin,
    # each branch a ladder of N pi-segments ending at the sink pin.
    N = 64
    r, c = nl.r_per_um, nl.c_per_um
    px = nl.x.astype(float)[nl.pin_cell] + nl.pin_dx
    py = nl.y.astype(float)[nl.pin_cell] + nl.pin_dy
    parent, R, Cn = [-1, 0], [0.0, float(nl.cell_rdrv[0])], [0.0, 0.0]
    sink_node = {}
    for s in range(1, fan + 1):
        L = abs(px[s] - px[0]) + abs(py[s] - py[0])
        prev = 1
        for k in range(N):
            parent.append(prev)
            R.append(r * L / N)
            Cn.append(0.0)
            cur = len(parent) - 1
            Cn[prev] += c * L / N / 2          # pi segment: half at each end
            Cn[cur] += c * L / N / 2
            prev = cur
        Cn[prev] += float(nl.pin_cap[s])
        sink_node[s] = prev
    delay = _elmore_tree(parent, R, Cn)
    for s, node in sink_node.items():
        expect = (tm["dnet"][0] - nl.d0_ps) + tm["tnet"][s]
        assert delay[node] == pytest.approx(expect, rel=1e-12)


# ----------------------------------------------------------- brute force ----

def _in_arcs(nl, tm):
    """In-arcs of every pin: (from_pin, delay); launch delay of startpoints."""
    pin_net = np.repeat(np.arange(nl.n_nets), np.diff(nl.net_ptr))
    drv = nl.net_ptr[:-1]
    cell_in = {}
    cell_out = {}
    for p in range(nl.n_pins):
        c = int(nl.pin_cell[p])
        if nl.pin_dir[p] == 1:
            cell_out[c] = p
        else:
            cell_in.setdefault(c, []).append(p)
    arcs, launch = {}, {}
    for p in range(nl.n_pins):
        c = int(nl.pin_cell[p])
        t = nl.cell_type[c]
        if nl.pin_dir[p] == 0:
            arcs[p] = [(int(drv[pin_net[p]]), tm["tnet"][p])]
        elif t == netgen.COMB:
            arcs[p] = [(i, tm["dnet"][pin_net[p]]) for i in cell_in[c]]
        else:
            launch[p] = tm["dnet"][pin_net[p]]
    return arcs, launch


def _all_paths(arcs, launch, ep):
    """Every path ending at ep: (delay summed start -> end, pins start first)."""
    out = []

    def rec(v, suffix):
        if v in launch:
            pins = [v] + suffix
            d = launch[v]
            for a, b in zip(pins[:-1], pins[1:]):
                d += dict(arcs[b])[a] if len(arcs[b]) == 1 else next(dl for u, dl in arcs[b] if u == a)
            out.append((d, pins))
            return
        for u, _ in arcs[v]:
            rec(u, [v] + suffix)

    rec(ep, [])
    return out


@pytest.mark.parametrize("seed", range(1, 9))
@pytest.mark.parametrize("keep_nonneg", [False, True])
def test_topk_equals_brute_force(seed, keep_nonneg):
    nl = netgen.generate(SMALL, seed)
    T = oracle.clock_period(nl, SMALL.t_factor)
    tm = oracle.sta(nl, T=T)
    K = SMALL.K
    P = oracle.topk(nl, tm, -1, K, keep_nonneg)
    arcs, launch = _in_arcs(nl, tm)
    eps_tol = 1e-9
    for ep in P["viol"]:
        bf = [(T - d, pins) for d, pins in _all_paths(arcs, launch, int(ep))]
        assert len(bf) < 100_000
        # slack ascending, then the pin sequence read from the endpoint backwards
        bf.sort(key=lambda t: (t[0], t[1][::-1]))
        if not keep_nonneg:
            bf = [t for t in bf if t[0] < 0]
        mine = [(P["slack"][k], P["pins"][P["pin_ptr"][k]:P["pin_ptr"][k + 1]].tolist())
                for k in np.nonzero(P["ep"] == ep)[0]]
        exp = bf[:K]
        assert len(mine) == len(exp)
        np.testing.assert_allclose([m[0] for m in mine], [e[0] for e in exp], atol=eps_tol)
        # compare sequences where the order is not decided by rounding-level gaps
        for k, (m, e) in enumerate(zip(mine, exp)):
            near = [t for t in bf if abs(t[0] - e[0]) <= eps_tol]
            if len(near) == 1:
                assert m[1] == e[1]
            else:
                assert m[1] in [t[1] for t in near]


def test_brute_force_counts_all_violating_endpoints():
    nl = netgen.generate(SMALL, 4)
    T = oracle.clock_period(nl, SMALL.t_factor)
    tm = oracle.sta(nl, T=T)
    ct = nl.cell_type[nl.pin_cell]
    ep = np.nonzero((nl.pin_dir == 0) & ((ct == netgen.FF) | (ct == netgen.PO)))[0]
    viol = ep[(T - tm["arr"][ep]) < 0]
    P = oracle.topk(nl, tm, -1, 1)
    assert sorted(P["viol"].tolist()) == sorted(viol.tolist())
    s = T - tm["arr"][P["viol"]]
    order = np.lexsort((P["viol"], s))
    np.testing.assert_array_equal(P["viol"][order], P["viol"])


# ------------------------------------------------------------ invariants ----

def _endpoints(nl):
    ct = nl.cell_type[nl.pin_cell]
    return np.nonzero((nl.pin_dir == 0) & ((ct == netgen.FF) | (ct == netgen.PO)))[0]


@pytest.mark.parametrize("cfg,seed", [("tiny", 1), ("tiny", 2), ("diff", 1)])
def test_sta_invariants(cfg, seed):
    nl = netgen.generate(cfg, seed)
    T = oracle.clock_period(nl, netgen.CONFIGS[cfg].t_factor)
    tm = oracle.sta(nl, T=T)
    ep = _endpoints(nl)
    s = T - tm["arr"][ep]
    assert tm["wns"] == pytest.approx(min(0.0, s.min()), abs=1e-9)
    assert tm["tns"] == pytest.approx(s[s < 0].sum(), rel=1e-12)
    assert tm["slack"].min() == pytest.approx(tm["wns"], abs=1e-7)
    np.testing.assert_allclose(tm["slack"][ep], s, atol=1e-9)
    # translation invariance
    sh = oracle.sta(nl, nl.x.astype(float) + 123.25, nl.y.astype(float) - 77.5, T)
    np.testing.assert_allclose(sh["arr"], tm["arr"], atol=1e-7)
    np.testing.assert_allclose(sh["slack"], tm["slack"], atol=1e-7)
    # paths: rank-1 slack = endpoint slack, non-decreasing with rank,
    # and every pin on a path has slack <= the path slack
    K = netgen.CONFIGS[cfg].K
    P = oracle.topk(nl, tm, -1, K)
    for k in range(len(P["slack"])):
        pins = P["pins"][P["pin_ptr"][k]:P["pin_ptr"][k + 1]]
        assert pins[-1] == P["ep"][k]
        assert (tm["slack"][pins] <= P["slack"][k] + 1e-7).all()
        if P["rank"][k] == 0:
            assert P["slack"][k] == pytest.approx(tm["slack"][P["ep"][k]], abs=1e-7)
        else:
            assert P["slack"][k] >= P["slack"][k - 1] - 1e-9
    # the WNS endpoint's worst path has slack = WNS at every pin
    k0 = int(np.nonzero((P["ep"] == P["viol"][0]) & (P["rank"] == 0))[0][0])
    pins = P["pins"][P["pin_ptr"][k0]:P["pin_ptr"][k0 + 1]]
    np.testing.assert_allclose(tm["slack"][pins], tm["wns"], atol=1e-7)


# ---------------------------------------------------------- pair update ----

@pytest.mark.parametrize("seed", [1, 2])
def test_pair_update_closed_form(seed):
    nl = netgen.generate("tiny", seed)
    T = oracle.clock_period(nl, 0.9)
    tm = oracle.sta(nl, T=T)
    P = oracle.topk(nl, tm, -1, 4)
    w0, w1, wns = 10.0, 0.2, tm["wns"]
    # a prior state: a random subset of sinks already in P with random weights
    rng = np.random.default_rng(seed)
    prior = (nl.pin_dir == 0) & (rng.random(nl.n_pins) < 0.3)
    w_prior = np.where(prior, rng.uniform(5, 20, nl.n_pins), 0.0)
    in_p, w = oracle.update_pairs(nl, P, wns, w0, w1, prior.astype(np.uint8), w_prior)
    ssum = np.zeros(nl.n_pins)
    smin = np.full(nl.n_pins, np.inf)
    for k in range(len(P["slack"])):
        pins = P["pins"][P["pin_ptr"][k]:P["pin_ptr"][k + 1]]
        sinks = pins[1::2]                     # start(drv), sink, out(drv), sink, ...
        assert (nl.pin_dir[sinks] == 0).all() and (nl.pin_dir[pins[0::2]] == 1).all()
        ssum[sinks] += P["slack"][k]
        smin[sinks] = np.minimum(smin[sinks], P["slack"][k])
    touched = np.isfinite(smin)
    exp_w = w_prior.copy()
    new = touched & ~prior
    old = touched & prior
    exp_w[new] = w0 + (w1 / wns) * (ssum[new] - smin[new])
    exp_w[old] = w_prior[old] + (w1 / wns) * ssum[old]
    np.testing.assert_array_equal(in_p.astype(bool), prior | touched)
    np.testing.assert_allclose(w, exp_w, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------ loss ----

def _pairs(nl, seed):
    rng = np.random.default_rng(seed)
    in_p = ((nl.pin_dir == 0) & (rng.random(nl.n_pins) < 0.4)).astype(np.uint8)
    w = np.where(in_p > 0, rng.uniform(5, 20, nl.n_pins), 0.0)
    return in_p, w


@pytest.mark.parametrize("seed", [1, 2])
def test_loss_central_differences(seed):
    nl = netgen.generate("tiny", seed)
    in_p, w = _pairs(nl, seed)
    x, y = nl.x.astype(float), nl.y.astype(float)
    pp, gx, gy = oracle.loss(nl, in_p, w, 2.5e-5, x, y, drop_fixed=False)
    rng = np.random.default_rng(seed)
    # PP is quadratic, so central differences are exact for any step up to
    # rounding of PP itself (~1e-15 |PP| per evaluation)
    h = 0.5
    tol = 1e-13 * abs(pp) / h
    for c in rng.choice(nl.n_cells, 40, replace=False):
        for arr_, g in ((x, gx), (y, gy)):
            a = arr_.copy()
            a[c] += h
            lp = oracle.loss(nl, in_p, w, 2.5e-5, a if arr_ is x else x, a if arr_ is y else y)[0]
            a[c] -= 2 * h
            lm = oracle.loss(nl, in_p, w, 2.5e-5, a if arr_ is x else x, a if arr_ is y else y)[0]
            assert (lp - lm) / (2 * h) == pytest.approx(g[c], rel=1e-9, abs=tol)


def test_loss_translation_and_euler():
    nl = netgen.generate("tiny", 5)          # zero pin offsets in this configuration
    assert not nl.pin_dx.any() and not nl.pin_dy.any()
    in_p, w = _pairs(nl, 5)
    x, y = nl.x.astype(float), nl.y.astype(float)
    pp, gx, gy = oracle.loss(nl, in_p, w, 1.0, x, y, drop_fixed=False)
    assert abs(gx.sum()) < 1e-6 * np.abs(gx).sum()
    assert abs(gy.sum()) < 1e-6 * np.abs(gy).sum()
    assert (x * gx + y * gy).sum() == pytest.approx(2 * pp, rel=1e-10)
    pp2 = oracle.loss(nl, in_p, w, 1.0, x + 17.0, y - 3.0)[0]
    assert pp2 == pytest.approx(pp, rel=1e-12)
    # fixed cells get no gradient when dropped
    _, gxd, gyd = oracle.loss(nl, in_p, w, 1.0, x, y, drop_fixed=True)
    assert not gxd[nl.cell_fixed > 0].any() and not gyd[nl.cell_fixed > 0].any()
    mv = nl.cell_fixed == 0
    np.testing.assert_array_equal(gxd[mv], gx[mv])


# ---------------------------------------------------- loss variants -------

def test_loss_kinds_hand_pair():
    """One pair: driver at (0, 0), sink at (3, 4), w = 2, beta = 1.5."""
    cells = [{"type": "FF", "x": 0.0, "y": 0.0, "rdrv": 1.0}, {"type": "FF", "x": 3.0, "y": 4.0, "rdrv": 1.0}]
    nl = netgen.from_lists(cells, [[(0, 0.0), (1, 1.0)]])
    in_p = np.array([0, 1], np.uint8)
    w = np.array([0.0, 2.0])
    x, y = np.array([0.0, 3.0]), np.array([0.0, 4.0])
    exp = {"quadratic": (1.5 * 2 * 25, 1.5 * 2 * 2 * 3, 1.5 * 2 * 2 * 4),
           "hpwl": (1.5 * 2 * 7, 1.5 * 2 * 1, 1.5 * 2 * 1),
           "euclid": (1.5 * 2 * 5, 1.5 * 2 * 3 / 5, 1.5 * 2 * 4 / 5)}
    for kind, (pp_e, gxs, gys) in exp.items():
        pp, gx, gy = oracle.loss(nl, in_p, w, 1.5, x, y, drop_fixed=False, kind=kind)
        assert pp == pytest.approx(pp_e, rel=1e-15)
        np.testing.assert_allclose(gx, [-gxs, gxs], rtol=1e-15)
        np.testing.assert_allclose(gy, [-gys, gys], rtol=1e-15)
    # coinciding pins: distance 0, gradient 0 for the non-smooth kinds
    for kind in ("hpwl", "euclid"):
        pp, gx, gy = oracle.loss(nl, in_p, w, 1.5, np.zeros(2), np.zeros(2), drop_fixed=False, kind=kind)
        assert pp == 0.0 and not gx.any() and not gy.any()


@pytest.mark.parametrize("kind", ["hpwl", "euclid"])
def test_loss_kinds_euler_translation_differences(kind):
    nl = netgen.generate("tiny", 6)          # zero pin offsets
    in_p, w = _pairs(nl, 6)
    x, y = nl.x.astype(float), nl.y.astype(float)
    pp, gx, gy = oracle.loss(nl, in_p, w, 1.0, x, y, drop_fixed=False, kind=kind)
    # degree 1: sum(x dPP/dx + y dPP/dy) = PP; translation invariance
    assert (x * gx + y * gy).sum() == pytest.approx(pp, rel=1e-10)
    assert abs(gx.sum()) < 1e-9 * np.abs(gx).sum() and abs(gy.sum()) < 1e-9 * np.abs(gy).sum()
    assert oracle.loss(nl, in_p, w, 1.0, x + 11.0, y - 5.0, kind=kind)[0] == pytest.approx(pp, rel=1e-12)
    # central differences on cells whose pairs stay away from dx = 0 / dy = 0
    h = 1e-4
    pc, nptr = nl.pin_cell, nl.net_ptr
    near = np.zeros(nl.n_cells, bool)
    for e in range(nl.n_nets):
        d = nptr[e]
        for s_ in range(d + 1, nptr[e + 1]):
            if in_p[s_] and (abs(x[pc[s_]] - x[pc[d]]) < 10 * h or abs(y[pc[s_]] - y[pc[d]]) < 10 * h):
                near[pc[s_]] = near[pc[d]] = True
    rng = np.random.default_rng(6)
    cand = np.nonzero(~near)[0]
    for c in rng.choice(cand, 40, replace=False):
        for axis in (0, 1):
            xp, yp, xm, ym = x.copy(), y.copy(), x.copy(), y.copy()
            (xp if axis == 0 else yp)[c] += h
            (xm if axis == 0 else ym)[c] -= h
            fd = (oracle.loss(nl, in_p, w, 1.0, xp, yp, kind=kind)[0] -
                  oracle.loss(nl, in_p, w, 1.0, xm, ym, kind=kind)[0]) / (2 * h)
            g = (gx if axis == 0 else gy)[c]
            assert fd == pytest.approx(g, rel=1e-5, abs=1e-9 * pp / h)


# ------------------------------------------------------- report_timing(n) ----

@pytest.mark.parametrize("seed", [1, 2, 3, 5])
@pytest.mark.parametrize("keep_nonneg", [False, True])
@pytest.mark.parametrize("n", [1, 6, 45, 100_000])
def test_report_timing_equals_brute_force(seed, keep_nonneg, n):
    """report_timing(n): the n lowest-slack paths over every endpoint of the
    design, brute force over all paths (n = 100000 exceeds their number)."""
    nl = netgen.generate(SMALL, seed)
    T = oracle.clock_period(nl, SMALL.t_factor)
    tm = oracle.sta(nl, T=T)
    arcs, launch = _in_arcs(nl, tm)
    bf = []
    for ep in _endpoints(nl):
        bf += [(T - d, pins) for d, pins in _all_paths(arcs, launch, int(ep))]
    assert len(bf) < 200_000
    bf.sort(key=lambda t: (t[0], t[1][::-1]))
    if not keep_nonneg:
        bf = [t for t in bf if t[0] < 0]
    exp = bf[:n]
    R = oracle.report_timing(nl, tm, n, keep_nonneg)
    mine = [(R["slack"][k], R["pins"][R["pin_ptr"][k]:R["pin_ptr"][k + 1]].tolist()) for k in range(len(R["ep"]))]
    assert len(mine) == len(exp)
    tol = 1e-9
    np.testing.assert_allclose([m[0] for m in mine], [e[0] for e in exp], atol=tol)
    for m, e in zip(mine, exp):
        assert m[1][-1] == R["ep"][mine.index(m)]
        near = [t[1] for t in bf if abs(t[0] - e[0]) <= tol]
        if len(near) == 1:
            assert m[1] == e[1]
        else:
            assert m[1] in near


def test_report_timing_small_cases():
    nl = netgen.generate(SMALL, 4)
    T = oracle.clock_period(nl, SMALL.t_factor)
    tm = oracle.sta(nl, T=T)
    assert len(oracle.report_timing(nl, tm, 0)["ep"]) == 0
    # n = 1: the worst path of the most critical endpoint
    R1 = oracle.report_timing(nl, tm, 1)
    P1 = oracle.topk(nl, tm, 1, 1)
    assert R1["ep"].tolist() == P1["ep"].tolist()
    assert R1["pins"].tolist() == P1["pins"].tolist()
    # nothing fails at a large clock period, unless non-negative paths are kept
    tm2 = oracle.sta(nl, T=10 * T)
    assert len(oracle.report_timing(nl, tm2, 50)["ep"]) == 0
    assert len(oracle.report_timing(nl, tm2, 50, keep_nonneg=True)["ep"]) == 50
    with pytest.raises(ValueError):
        oracle.report_timing(nl, tm, -1)


def test_report_timing_spreads_over_endpoints():
    """Eight one-path chains PI -> buffer -> PO of different lengths and one
    PO behind a 3-input cell (three paths): at T = 0 every path fails, and
    report_timing(n) must list the n lowest slacks over all nine endpoints --
    n distinct endpoints when the chains are the most critical."""
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
    tm = oracle.sta(nl, T=0.0)
    arcs, launch = _in_arcs(nl, tm)
    bf = sorted((-d, pins[-1]) for ep in _endpoints(nl) for d, pins in _all_paths(arcs, launch, int(ep)))
    assert len(bf) == 11
    for n in (1, 4, 8, 11):
        R = oracle.report_timing(nl, tm, n)
        assert len(R["ep"]) == n
        np.testing.assert_allclose(R["slack"], [t[0] for t in bf[:n]], atol=1e-9)
        assert sorted(R["ep"].tolist()) == sorted(t[1] for t in bf[:n])
    # the 8 worst paths end at more than 4 different endpoints
    assert len(set(t[1] for t in bf[:8])) > 4
