"""Helpers for comparing the CUDA library with the FP64 oracle.

Tolerances (stated per result), |d| <= 1e-3 ps + 1e-6 * scale, where the
scale is the magnitude of the delay sum that produced the value (FP32 delays
each carry a relative rounding error, so the error grows with the sum, not
with the difference T - sum):
* net delay, load, cell delay: the value itself;
* arrival time: |arr| (a sum of positive delays);
* required time: max(|req|, T - req) (T minus the suffix delay);
* slack: max(|arr|, |req|, T - slack) (T - slack is the delay of the worst
  path through the pin);
* FP64-on-GPU vs the oracle: 1e-7 ps + 1e-11 |ref| (same arithmetic, other
  operation order and fused multiply-adds);
* extracted path sets: identical pin sequences on every endpoint whose
  top-K set is decided by more than the slack tolerance (its slack, the gap
  between the K-th and (K+1)-th path, and, when only negative paths are kept,
  the margin of the boundary path to zero).
"""
import numpy as np
import torch

import oracle

TOL32 = (1e-3, 1e-6)
TOL64 = (1e-7, 1e-11)


def tol_of(dtype):
    return TOL32 if dtype == torch.float32 else TOL64


def close(got, ref, scale, tol):
    a, r = tol
    return np.abs(got - ref) <= a + r * np.abs(scale)


def sta_scales(tm, T):
    """Scales of the relative tolerance term for arr, req and slack."""
    arr, req, sl = tm["arr"], tm["req"], tm["slack"]
    s_arr = np.abs(arr)
    s_req = np.maximum(np.abs(req), T - req)
    s_sl = np.maximum.reduce([np.abs(arr), np.abs(req), T - sl])
    return s_arr, s_req, s_sl


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def check_sta(G, tm, T, tol):
    """Net delays and per-pin arr / req / slack of the graph against the oracle."""
    tnet, cload, dnet = (_np(t) for t in G.sta_get_net_delays())
    for got, key in ((tnet, "tnet"), (cload, "cload"), (dnet, "dnet")):
        ok = close(got, tm[key], tm[key], tol)
        assert ok.all(), (key, np.abs(got - tm[key]).max())
    arr, req, slack = (_np(t) for t in G.sta_get_timing())
    s_arr, s_req, s_sl = sta_scales(tm, T)
    for got, key, sc in ((arr, "arr", s_arr), (req, "req", s_req), (slack, "slack", s_sl)):
        ok = close(got, tm[key], sc, tol)
        assert ok.all(), (key, np.abs(got - tm[key]).max(), int((~ok).sum()))
    return arr, req, slack


def check_net_weights(nl, tm, T, w_gpu, w_ref, n_gpu, n_ref, tol, eps, k, gamma):
    """Net weights after k updates against the oracle's (bound derived in
    tests/test_gpu_net_weights.py): |dw| <= gamma (tol_s + tol_WNS) / |WNS|
    + k x 4 rounding units x (1 + gamma); the counts of critical nets differ
    by at most the nets whose slack is within tol_s of zero."""
    a, r = tol
    drv = np.asarray(nl.net_ptr)[:-1]
    sc = sta_scales(tm, T)[2]
    tol_s = a + r * sc[drv]
    ct = nl.cell_type[nl.pin_cell]
    ep = np.nonzero((nl.pin_dir == 0) & ((ct == 1) | (ct == 3)))[0]
    tol_wns = a + r * sc[ep].max()
    dc = (tol_s + tol_wns) / max(abs(tm["wns"]), 1e-30)
    bound = gamma * dc + k * 4 * eps * (1 + gamma)
    err = np.abs(w_gpu - w_ref)
    assert (err <= bound).all(), (err.max(), int(np.argmax(err - bound)))
    near0 = int((np.abs(tm["slack"][drv]) <= tol_s).sum())
    assert abs(n_gpu - n_ref) <= near0, (n_gpu, n_ref, near0)


def paths_by_endpoint(P):
    """{endpoint: [(slack, pins tuple), ...] in rank order}."""
    out = {}
    ep = np.asarray(P["ep"])
    sl = np.asarray(P["slack"])
    ptr = np.asarray(P["pin_ptr"])
    pins = np.asarray(P["pins"])
    for k in range(len(ep)):
        out.setdefault(int(ep[k]), []).append((float(sl[k]), tuple(pins[ptr[k]:ptr[k + 1]].tolist())))
    return out


def gpu_paths(g):
    P = g.sta_get_paths()
    return {k: v.cpu().numpy() for k, v in P.items()}


def _pin_net(nl):
    npt = np.asarray(nl.net_ptr, dtype=np.int64)
    return np.repeat(np.arange(nl.n_nets, dtype=np.int64), np.diff(npt))


def path_checks(nl, tm, T, ptr, pins, ep):
    """Per path: whether the pin sequence is a path of the timing graph that
    ends at its endpoint (startpoint driver first, then sink / driver pairs
    joined by net arcs and cell arcs), and its slack recomputed in FP64 from
    the oracle's timing: T - (launch arrival + Elmore delays of its sinks +
    delays of the cells it crosses).  ``ptr`` / ``pins`` / ``ep`` are one
    chunk of paths (ptr relative to ``pins``)."""
    pin_net = _pin_net(nl)
    pin_dir = np.asarray(nl.pin_dir)
    pin_cell = np.asarray(nl.pin_cell)
    ctype = np.asarray(nl.cell_type)
    ptr = np.asarray(ptr, dtype=np.int64)
    pins = np.asarray(pins, dtype=np.int64)
    n = len(ptr) - 1
    ln = np.diff(ptr)
    ok = (ln >= 2) & (ln % 2 == 0)
    if n == 0:
        return ok, np.zeros(0)
    pid = np.repeat(np.arange(n), ln)
    pos = np.arange(len(pins)) - np.repeat(ptr[:-1], ln)
    even = pos % 2 == 0
    bad = np.zeros(n, bool)
    # even positions are drivers, odd positions sinks
    np.logical_or.at(bad, pid, (pin_dir[pins] == 1) != even)
    # sink 2i+1 lies on the net driven by pin 2i (a net arc)
    nxt = np.ones(len(pins), bool)
    nxt[ptr[1:] - 1] = False                    # last pin of a path has no successor
    a = np.nonzero(even & nxt)[0]
    np.logical_or.at(bad, pid[a], pin_net[pins[a]] != pin_net[pins[a + 1]])
    # sink 2i+1 and driver 2i+2 are pins of one combinational cell (a cell arc)
    b = np.nonzero(~even & nxt)[0]
    np.logical_or.at(bad, pid[b], (pin_cell[pins[b]] != pin_cell[pins[b + 1]])
                     | (ctype[pin_cell[pins[b]]] != 0))
    first = pins[ptr[:-1]]
    last = pins[ptr[1:] - 1]
    start_ok = np.isin(ctype[pin_cell[first]], (1, 2)) & (pin_dir[first] == 1)
    ok &= ~bad & start_ok & (last == np.asarray(ep))
    d = np.where(even, 0.0, tm["tnet"][pins])
    d += np.where(even & (pos > 0), tm["dnet"][pin_net[pins]], 0.0)
    arr = tm["arr"][first] + np.bincount(pid, weights=d, minlength=n)
    return ok, T - arr


def path_sinks(P, endpoints=None):
    """Sink pins (odd positions: the pins net arcs end on) of the paths of
    ``endpoints`` (all paths if None), with repetition."""
    ptr = np.asarray(P["pin_ptr"], dtype=np.int64)
    pins = np.asarray(P["pins"])
    sel = np.arange(len(ptr) - 1)
    if endpoints is not None:
        sel = np.nonzero(np.isin(np.asarray(P["ep"]), np.asarray(list(endpoints), dtype=np.int64)))[0]
    if len(sel) == 0:
        return np.zeros(0, np.int64)
    ln = ptr[sel + 1] - ptr[sel]
    pos = np.arange(int(ln.sum())) - np.repeat(np.cumsum(ln) - ln, ln)
    flat = np.repeat(ptr[sel], ln) + pos
    return pins[flat[pos % 2 == 1]].astype(np.int64)


def _group(ep):
    """{endpoint: (first, last + 1)} of a path array sorted by endpoint blocks."""
    ep = np.asarray(ep)
    if len(ep) == 0:
        return {}
    cut = np.nonzero(np.diff(ep))[0] + 1
    lo = np.concatenate([[0], cut])
    hi = np.concatenate([cut, [len(ep)]])
    return {int(ep[i]): (int(i), int(j)) for i, j in zip(lo, hi)}


def compare_paths(nl, tm, T, K, keep_nonneg, gpu, tol, endpoints=None, extra=8, chunk=4096,
                  detail=False):
    """Compare the GPU's extracted paths with the oracle's, endpoint by endpoint.

    ``gpu`` is the dict of sta_get_paths.  Endpoints: ``endpoints`` if given,
    else every endpoint either side reports as failing.  The oracle searches
    the K + ``extra`` best paths of each (any slack).

    Decided endpoints (R14: the endpoint slack, the gap between the K-th and
    the next path and, when only negative paths are kept, the boundary path's
    margin to zero all exceed the slack tolerance) must match bit-exactly:
    the same pin sequences, slacks within tolerance, and the same order
    wherever neighbouring slacks are separated.

    The others are ambiguous; there what is unique is compared and the rest
    checked for validity: every GPU path is a path of the timing graph ending
    at the endpoint, with its slack equal (within tolerance) to the one the
    oracle's timing gives its pin sequence; no sequence repeats; every oracle
    path better than the cut by more than the tolerance is reported; no
    reported path is worse, beyond the tolerance, than an oracle path left
    out; the count lies between the counts the tolerance band allows; slacks
    are non-decreasing within tolerance.

    Returns (n_checked, n_ambiguous), or with ``detail`` a dict that also
    holds the endpoints whose sets differ (all ambiguous), the largest
    |slack - oracle slack| over the compared paths, and the path count.
    """
    a, r = tol
    gep = np.asarray(gpu["ep"])
    gsl = np.asarray(gpu["slack"], dtype=np.float64)
    gptr = np.asarray(gpu["pin_ptr"], dtype=np.int64)
    gpins = np.asarray(gpu["pins"])
    got = _group(gep)
    if endpoints is None:
        ct = np.asarray(nl.cell_type)[np.asarray(nl.pin_cell)]
        ep_all = np.nonzero((np.asarray(nl.pin_dir) == 0) & ((ct == 1) | (ct == 3)))[0]
        ref_fail = ep_all[tm["slack"][ep_all] < 0.0]
        eps = np.union1d(np.asarray(gpu["viol"]), ref_fail).astype(np.int64)
    else:
        eps = np.asarray(endpoints, dtype=np.int64)
    checked = ambiguous = 0
    differ, max_err, n_cmp = [], 0.0, 0
    for c0 in range(0, len(eps), chunk):
        ce = eps[c0:c0 + chunk]
        ref = oracle.topk(nl, tm, -1, K + extra, True, endpoints=ce)
        rby = _group(ref["ep"])
        rsl, rptr, rpins = ref["slack"], ref["pin_ptr"], ref["pins"]
        # the GPU paths of this chunk, validated and re-timed in one pass
        idx = np.concatenate([np.arange(*got[int(e)]) for e in ce if int(e) in got] or
                             [np.zeros(0, np.int64)]).astype(np.int64)
        lens = gptr[idx + 1] - gptr[idx]
        sub_ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        sub_pins = np.concatenate([gpins[gptr[k]:gptr[k + 1]] for k in idx] or [np.zeros(0, np.int32)])
        valid, rs = path_checks(nl, tm, T, sub_ptr, sub_pins, gep[idx])
        row = {int(k): i for i, k in enumerate(idx)}
        for e in ce:
            e = int(e)
            lo_r, hi_r = rby.get(e, (0, 0))
            full = [(float(rsl[k]), rpins[rptr[k]:rptr[k + 1]].tobytes()) for k in range(lo_r, hi_r)]
            tolp = a + r * (T + abs(full[0][0]) if full else T)
            exp = full[:K]
            if not keep_nonneg:
                exp = [p for p in exp if p[0] < 0]
            lo_g, hi_g = got.get(e, (0, 0))
            mine = [(float(gsl[k]), gpins[gptr[k]:gptr[k + 1]].tobytes(), k) for k in range(lo_g, hi_g)]
            nxt = full[len(exp)] if len(full) > len(exp) else None
            robust = abs(tm["slack"][e]) > tolp
            if nxt is not None and exp:
                robust &= nxt[0] - exp[-1][0] > tolp
            if not keep_nonneg and exp:
                robust &= exp[-1][0] < -tolp
            if not keep_nonneg and nxt is not None and len(exp) < K:
                robust &= nxt[0] > tolp
            mset = {p[1] for p in mine}
            assert len(mset) == len(mine), ("repeated path", e)
            sl = [p[0] for p in mine]
            assert all(sl[i] <= sl[i + 1] + tolp for i in range(len(sl) - 1)), ("order", e)
            for s, _, k in mine:
                i = row[k]
                assert valid[i], ("not a path of the timing graph", e, k)
                assert abs(s - rs[i]) <= tolp, ("slack of the pin sequence", e, s, rs[i])
                if not keep_nonneg:
                    assert rs[i] < tolp, ("non-negative path kept", e, rs[i])
                max_err = max(max_err, abs(s - rs[i]))
            n_cmp += len(mine)
            if robust:
                checked += 1
                assert len(mine) == len(exp), (e, len(mine), len(exp))
                assert mset == {p[1] for p in exp}, ("path set", e)
                # order: where neighbouring oracle slacks are separated, the order matches
                for i in range(len(exp)):
                    sep_prev = i == 0 or exp[i][0] - exp[i - 1][0] > tolp
                    sep_next = i == len(exp) - 1 or exp[i + 1][0] - exp[i][0] > tolp
                    if sep_prev and sep_next:
                        assert mine[i][1] == exp[i][1], ("order", e, i)
                continue
            ambiguous += 1
            if mset != {p[1] for p in exp}:
                differ.append(e)
            # the cut: the K-th path's slack when K qualify, else zero (or
            # every path, keep_nonneg); paths better than it beyond the
            # tolerance are unique to the answer
            cut = exp[-1][0] if len(exp) == K else (0.0 if not keep_nonneg else np.inf)
            for s, seq in full:
                if s < cut - tolp:
                    assert seq in mset, ("missing path", e, s)
            left_out = [s for s, seq in full if seq not in mset]
            if left_out and mine:
                assert max(sl) <= min(left_out) + tolp, ("worse path reported", e)
            if len(full) == K + extra and mine:
                assert max(sl) <= full[-1][0] + tolp, ("worse path reported", e)
            if keep_nonneg:
                n_lo = min(K, len(full))
                n_hi = K
            else:
                n_lo = min(K, sum(1 for s, _ in full if s < -tolp))
                below = sum(1 for s, _ in full if s < tolp)
                n_hi = K if below == len(full) else min(K, below)
            assert n_lo <= len(mine) <= n_hi, ("count", e, len(mine), n_lo, n_hi)
    if detail:
        return {"checked": checked, "ambiguous": ambiguous, "differ": differ,
                "max_slack_err": max_err, "paths": n_cmp}
    return checked, ambiguous
