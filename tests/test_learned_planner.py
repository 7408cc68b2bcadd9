"""Host side of the learned planner: the a-priori key set covers every
candidate plan, and the features are a function of the plan."""
import numpy as np

import paper_2506_10399_gb300 as fg
from paper_2506_10399_gb300 import learn_planner as lp
from paper_2506_10399_gb300 import workloads as wl


def test_key_set_covers_every_candidate_plan():
    P = wl.BATCH_PARAMS
    M = 1 << (P["log_n"] - 1)
    allam = lp.all_amounts(M)
    for s in (2000, 1003):
        w = wl.planner_graphs([s])[0]
        t_rule = lp.packing_t(fg, P, w)
        for c in lp.CANDIDATES:
            t = lp.candidate_t(c, t_rule, w.V, M)
            if t is None:
                continue
            perm = lp.candidate_perm(fg, wl, w, M // t, c, s)
            rec = fg.plan_dry_run(P, w.row_ptr, w.col, w.val, w.W, perm, t=t, radix_bits=c["radix_bits"])
            assert lp._record_amounts(rec, M) <= allam
            f = fg.plan_features(P, w.row_ptr, w.col, w.val, w.W, perm, t=t, radix_bits=c["radix_bits"])
            assert f[5] == c["radix_bits"] and f[7] == rec[11] and round(2 ** f[4]) == t


def test_features_follow_the_order():
    """NOO places neighbours close: shorter shifts than a random order."""
    P = wl.BATCH_PARAMS
    M = 1 << (P["log_n"] - 1)
    w = wl.planner_graphs([1005])[0]
    t = lp.packing_t(fg, P, w)
    fr = fg.plan_features(P, w.row_ptr, w.col, w.val, w.W,
                          lp.candidate_perm(fg, wl, w, M // t, lp.CANDIDATES[0], 1005), t=t, radix_bits=2)
    fn = fg.plan_features(P, w.row_ptr, w.col, w.val, w.W,
                          lp.candidate_perm(fg, wl, w, M // t, lp.CANDIDATES[5], 1005), t=t, radix_bits=2)
    assert fn[6] < fr[6]
    assert np.all(fr[:6] == fn[:6])


def _model():
    import json
    import os
    import pytest
    if not os.path.exists(lp.MODEL):
        pytest.skip("no trained model")
    return json.load(open(lp.MODEL))


def test_candidates_span_the_decisions():
    """t (rule and neighbour), radix (4, 8, 16), order (random, NOO with two
    region sizes and both region orders)."""
    ts = {c["t"] for c in lp.CANDIDATES}
    assert ts == {"rule", "alt"}
    assert {c["radix_bits"] for c in lp.CANDIDATES} == {2, 3, 4}
    noo = [c for c in lp.CANDIDATES if c["order"] == "noo"]
    assert {c["TH"] for c in noo} == {256, 1024} and {c["region_order"] for c in noo} == {0, 1}
    assert lp.CANDIDATES[lp.DEFAULT] == dict(radix_bits=2, order="random", t="rule")
    assert lp.candidate_t(lp.CANDIDATES[3], 4, 1500, 32768) == 1
    assert lp.candidate_t(lp.CANDIDATES[3], 1, 5000, 32768) == 2
    assert lp.candidate_t(lp.CANDIDATES[3], 1, 20000, 32768) is None


def test_trained_model_against_exhaustive_and_default():
    """What the trained latency model gains: on the 20 held-out graphs (seeds
    2000-2019, measured on a GB300), the candidates it picks (scored here
    with the FP64 reference forward pass on the model's own weights) against
    the exhaustive planner's fastest and the default plan (radix 4, random
    order, t by the rule).  The model must not lose to the default."""
    from oracle import mlp
    d = _model()
    rows = [r for r in lp.complete(lp.load(lp.DATA)) if r["seed"] in lp.HELD_OUT]
    assert len(rows) == 20
    params = mlp.unpack(np.array(d["params"], dtype=np.float64), d["n_in"], d["hidden"])
    mu, sd = np.array(d["mean"]), np.array(d["std"])
    chosen = best = default = 0.0
    for r in rows:
        F = (np.array([c["features"] for c in r["cands"]]) - mu) / sd
        f, _ = mlp.forward(params, F)
        ms = [c["ms"] for c in r["cands"]]
        chosen += ms[lp.pick(np.ravel(f), r["cands"], d["margin"])]
        best += min(ms)
        default += lp.default_ms(r)
    gap, gain = chosen / best - 1, 1 - chosen / default
    assert abs(gap - d["held_out"]["gap_vs_exhaustive"]) < 2e-3
    assert abs(gain - d["held_out"]["gain_vs_default"]) < 2e-3
    assert gain >= 0.0
    print("held-out: gain over the default %.4f, gap to the exhaustive planner %.4f" % (gain, gap))
