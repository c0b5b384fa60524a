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


def compare_paths(nl, tm, T, K, keep_nonneg, gpu, tol, endpoints=None):
    """Compare GPU paths with the oracle's; returns (n_checked, n_ambiguous).

    ``gpu`` is the dict of sta_get_paths; ``endpoints`` restricts the check.
    """
    a, r = tol
    ref_full = oracle.topk(nl, tm, -1, K + 1, True, endpoints=endpoints)   # K+1 best, any slack
    ref_full = paths_by_endpoint(ref_full)
    got = paths_by_endpoint(gpu)
    eps = list(ref_full) if endpoints is None else [int(e) for e in endpoints]
    checked = ambiguous = 0
    for e in eps:
        full = ref_full.get(e, [])
        tolp = a + r * (T + abs(full[0][0]) if full else T)
        exp = full[:K]
        if not keep_nonneg:
            exp = [p for p in exp if p[0] < 0]
        mine = got.get(e, [])
        # the boundary that decides the set
        nxt = full[len(exp)] if len(full) > len(exp) else None
        robust = abs(tm["slack"][e]) > tolp
        if nxt is not None and exp:
            robust &= nxt[0] - exp[-1][0] > tolp
        if not keep_nonneg and exp:
            robust &= exp[-1][0] < -tolp
        if not keep_nonneg and nxt is not None and len(exp) < K:
            robust &= nxt[0] > tolp
        if not robust:
            ambiguous += 1
            # still: same number of paths within one, and valid slacks
            assert abs(len(mine) - len(exp)) <= 1
            continue
        checked += 1
        assert len(mine) == len(exp), (e, len(mine), len(exp))
        assert set(p[1] for p in mine) == set(p[1] for p in exp), e
        ref_sl = {p[1]: p[0] for p in exp}
        for s, pins in mine:
            assert abs(s - ref_sl[pins]) <= tolp, (e, s, ref_sl[pins])
        sl = [p[0] for p in mine]
        assert all(sl[i] <= sl[i + 1] + tolp for i in range(len(sl) - 1))
        # order: where neighbouring oracle slacks are separated, the order matches
        for i in range(len(exp)):
            sep_prev = i == 0 or exp[i][0] - exp[i - 1][0] > tolp
            sep_next = i == len(exp) - 1 or exp[i + 1][0] - exp[i][0] > tolp
            if sep_prev and sep_next:
                assert mine[i][1] == exp[i][1]
    return checked, ambiguous
