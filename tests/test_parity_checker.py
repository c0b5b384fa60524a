"""The path-set comparison used by the GPU parity tests, checked on the CPU.

The oracle's own extraction must pass it with every endpoint compared, and
each plausible mistake of an extraction, planted in a copy of the oracle's
output, must fail it: a dropped path, a path of another endpoint, a pin
replaced, a slack off by a picosecond, two separated paths swapped, a path
repeated, a non-negative path kept.
"""
import numpy as np
import pytest

import netgen
import oracle
from parity_util import TOL32, compare_paths, path_checks

K = 4


@pytest.fixture(scope="module")
def case():
    nl = netgen.generate("tiny", 1)
    T = oracle.clock_period(nl, 0.9)
    tm = oracle.sta(nl, T=T)
    P = oracle.topk(nl, tm, -1, K, False)
    return nl, T, tm, P


def _copy(P):
    return {k: np.array(v, copy=True) for k, v in P.items()}


def _decided_endpoint_with(P, n_paths, tm, T):
    """An endpoint holding n_paths or more whose slacks are separated."""
    tolp = TOL32[0] + TOL32[1] * 2 * T
    ep = P["ep"]
    for e in P["viol"]:
        k = np.nonzero(ep == e)[0]
        if len(k) >= n_paths and (np.diff(P["slack"][k[:n_paths]]) > 2 * tolp).all() and tm["slack"][e] < -tolp:
            return int(e), k
    raise AssertionError("no such endpoint")


def _rebuild(P, keep):
    """P restricted to the path indices ``keep`` (in that order)."""
    lens = np.diff(P["pin_ptr"])[keep]
    return {"viol": P["viol"], "ep": P["ep"][keep], "slack": P["slack"][keep],
            "pin_ptr": np.concatenate([[0], np.cumsum(lens)]).astype(np.int64),
            "pins": np.concatenate([P["pins"][P["pin_ptr"][k]:P["pin_ptr"][k + 1]] for k in keep])}


def test_oracle_paths_pass_and_are_valid(case):
    nl, T, tm, P = case
    d = compare_paths(nl, tm, T, K, False, P, TOL32, detail=True)
    assert d["checked"] + d["ambiguous"] >= len(P["viol"])
    assert d["differ"] == [] and d["max_slack_err"] < 1e-6
    ok, rs = path_checks(nl, tm, T, P["pin_ptr"], P["pins"], P["ep"])
    assert ok.all()
    np.testing.assert_allclose(rs, P["slack"], atol=1e-6)


def test_keep_nonneg_oracle_paths_pass(case):
    nl, T, tm, _ = case
    P = oracle.topk(nl, tm, -1, K, True)
    d = compare_paths(nl, tm, T, K, True, P, TOL32, detail=True)
    assert d["differ"] == []


def test_dropped_path_fails(case):
    nl, T, tm, P = case
    e, k = _decided_endpoint_with(P, 2, tm, T)
    keep = np.setdiff1d(np.arange(len(P["ep"])), [k[1]])
    with pytest.raises(AssertionError):
        compare_paths(nl, tm, T, K, False, _rebuild(P, keep), TOL32)


def test_replaced_pin_fails(case):
    nl, T, tm, P = case
    Q = _copy(P)
    e, k = _decided_endpoint_with(P, 1, tm, T)
    s = Q["pin_ptr"][k[0]]
    # a sink pin of the path replaced by another sink of the same net would
    # still be connected one way; take a sink pin of a different net
    j = s + 1
    other = np.nonzero((nl.pin_dir == 0))[0]
    Q["pins"][j] = other[other != Q["pins"][j]][0]
    with pytest.raises(AssertionError):
        compare_paths(nl, tm, T, K, False, Q, TOL32)
    ok, _ = path_checks(nl, tm, T, Q["pin_ptr"], Q["pins"], Q["ep"])
    assert not ok[k[0]]


def test_slack_off_by_a_picosecond_fails(case):
    nl, T, tm, P = case
    Q = _copy(P)
    e, k = _decided_endpoint_with(P, 1, tm, T)
    Q["slack"][k[0]] += 1.0
    with pytest.raises(AssertionError):
        compare_paths(nl, tm, T, K, False, Q, TOL32)


def test_swapped_separated_paths_fail(case):
    nl, T, tm, P = case
    e, k = _decided_endpoint_with(P, 2, tm, T)
    order = np.arange(len(P["ep"]))
    order[k[0]], order[k[1]] = k[1], k[0]
    Q = _rebuild(P, order)
    with pytest.raises(AssertionError):
        compare_paths(nl, tm, T, K, False, Q, TOL32)


def test_path_of_another_endpoint_fails(case):
    nl, T, tm, P = case
    e, k = _decided_endpoint_with(P, 1, tm, T)
    other = int(np.nonzero(P["ep"] != e)[0][0])
    keep = np.arange(len(P["ep"]))
    keep[k[-1]] = other
    Q = _rebuild(P, keep)
    Q["ep"][k[-1]] = e
    with pytest.raises(AssertionError):
        compare_paths(nl, tm, T, K, False, Q, TOL32)


def test_repeated_path_fails(case):
    nl, T, tm, P = case
    e, k = _decided_endpoint_with(P, 2, tm, T)
    keep = np.arange(len(P["ep"]))
    keep[k[1]] = k[0]
    with pytest.raises(AssertionError):
        compare_paths(nl, tm, T, K, False, _rebuild(P, keep), TOL32)


def test_nonnegative_path_kept_fails(case):
    nl, T, tm, _ = case
    P = oracle.topk(nl, tm, -1, K, True)
    with pytest.raises(AssertionError):
        compare_paths(nl, tm, T, K, False, P, TOL32)


def test_path_sinks_are_the_odd_positions(case):
    from parity_util import path_sinks
    _, _, _, P = case
    want = np.concatenate([P["pins"][P["pin_ptr"][k]:P["pin_ptr"][k + 1]][1::2] for k in range(len(P["ep"]))])
    np.testing.assert_array_equal(path_sinks(P), want)
    e = int(P["viol"][3])
    ks = np.nonzero(P["ep"] == e)[0]
    want = np.concatenate([P["pins"][P["pin_ptr"][k]:P["pin_ptr"][k + 1]][1::2] for k in ks])
    np.testing.assert_array_equal(path_sinks(P, [e]), want)
    assert len(path_sinks(P, [])) == 0
