"""Pin the FP64 oracle to hand-computed circuits (tests/golden/*.json).

Each fixture states its derivation from Eq. (8), Section II-B, Eqs. (2)-(4),
report_timing_endpoint of Section III-B, Eq. (w_ij) and Eq. (9).
"""
import numpy as np
import pytest

import oracle
from golden_util import GOLDEN_NAMES, load

TOL = 1e-9


@pytest.mark.parametrize("name", GOLDEN_NAMES)
def test_sta_matches_hand_values(name):
    g, nl = load(name)
    e = g["expect"]
    tm = oracle.sta(nl, T=g["T"])
    for key in ("tnet", "arr", "req", "slack"):
        if key in e:
            np.testing.assert_allclose(tm[key], e[key], atol=TOL, rtol=0)
    for key in ("cload", "dnet"):
        if key in e:
            np.testing.assert_allclose(tm[key], e[key], atol=TOL, rtol=0)
    assert tm["wns"] == pytest.approx(e["wns"], abs=TOL)
    assert tm["tns"] == pytest.approx(e["tns"], abs=TOL)
    if "pred_of_G3_out" in e:
        assert tm["pred"][7] == e["pred_of_G3_out"]
    if "slack_G_b" in e:
        assert tm["slack"][3] == pytest.approx(e["slack_G_b"], abs=TOL)
        assert tm["slack"][5] == pytest.approx(e["slack_G_c"], abs=TOL)


def _paths_list(P):
    out = []
    for k in range(len(P["slack"])):
        pins = P["pins"][P["pin_ptr"][k]:P["pin_ptr"][k + 1]].tolist()
        out.append((int(P["ep"][k]), float(P["slack"][k]), pins))
    return out


@pytest.mark.parametrize("name", GOLDEN_NAMES)
def test_topk_matches_hand_paths(name):
    g, nl = load(name)
    tm = oracle.sta(nl, T=g["T"])
    got = _paths_list(oracle.topk(nl, tm, -1, g["K"]))
    exp = g["expect"]["paths"]
    assert len(got) == len(exp)
    for (ep, s, pins), ex in zip(got, exp):
        assert ep == ex["ep"] and pins == ex["pins"]
        assert s == pytest.approx(ex["slack"], abs=TOL)
    if "paths_keep_nonneg" in g["expect"]:
        got = _paths_list(oracle.topk(nl, tm, -1, g["K"], keep_nonneg=True))
        exp = g["expect"]["paths_keep_nonneg"]
        assert [p[2] for p in got] == [ex["pins"] for ex in exp]
        np.testing.assert_allclose([p[1] for p in got], [ex["slack"] for ex in exp], atol=TOL)


@pytest.mark.parametrize("name", GOLDEN_NAMES)
def test_pair_update_and_loss_match_hand_values(name):
    g, nl = load(name)
    e = g["expect"]
    tm = oracle.sta(nl, T=g["T"])
    P = oracle.topk(nl, tm, -1, g["K"])
    in_p, w = oracle.update_pairs(nl, P, tm["wns"], g["w0"], g["w1"])
    exp = {int(k): v for k, v in e["pairs_after_one_update"].items()}
    assert sorted(np.nonzero(in_p)[0].tolist()) == sorted(exp)
    for s, v in exp.items():
        assert w[s] == pytest.approx(v, abs=1e-12)
    pp, gx, gy = oracle.loss(nl, in_p, w, g["beta"])
    assert pp == pytest.approx(e["pp"], rel=1e-13)
    np.testing.assert_allclose(gx, e["gx"], atol=1e-9)
    np.testing.assert_allclose(gy, e["gy"], atol=1e-9)
    if "pairs_after_two_updates" in e:
        in_p2, w2 = oracle.update_pairs(nl, P, tm["wns"], g["w0"], g["w1"], in_p, w)
        for s, v in e["pairs_after_two_updates"].items():
            assert w2[int(s)] == pytest.approx(v, abs=1e-12)


def test_topk_limits_endpoint_count():
    """n most critical endpoints only (report_timing_endpoint(n, k))."""
    import netgen
    nl = netgen.generate("tiny", 3)
    T = oracle.clock_period(nl, 0.9)
    tm = oracle.sta(nl, T=T)
    allp = oracle.topk(nl, tm, -1, 2)
    three = oracle.topk(nl, tm, 3, 2)
    assert set(three["ep"].tolist()) == set(allp["viol"][:3].tolist())
    first = np.isin(allp["ep"], allp["viol"][:3])
    np.testing.assert_array_equal(three["slack"], allp["slack"][first])
