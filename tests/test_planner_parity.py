"""The library's host planner (C++) against the oracle's planner (Python):
identical plans, record for record -- rotations, lanes, masked products and
every mask value bit -- on the same seeded graphs and node orders.  Host
only: no GPU is used (fg_plan_dry_run)."""
import math

import numpy as np
import pytest

import paper_2506_10399_gb300 as fg
from oracle import ckks, planner
from paper_2506_10399_gb300 import workloads as wl
from plan_records import oracle_records

CASES = [
    # (params, workload, t, radix, aoo, order)
    (dict(log_n=10, q_bits=[60] + [40] * 12, p_bits=[60], alpha=1, log_scale=40),
     dict(graph="er", V=48, deg=4.0, F=5, Fp=3, seed=1), 1, 1, True, "random"),
    (dict(log_n=10, q_bits=[60] + [40] * 12, p_bits=[60], alpha=1, log_scale=40),
     dict(graph="er", V=48, deg=4.0, F=5, Fp=3, seed=1), 1, 2, False, "identity"),
    (dict(log_n=11, q_bits=[60] + [40] * 8, p_bits=[60, 60], alpha=2, log_scale=40),
     dict(graph="chung_lu", V=300, deg=4.0, gamma=2.2, F=7, Fp=4, x="tfidf", w="glorot", seed=2),
     1, 3, True, "random"),
    (dict(log_n=11, q_bits=[60] + [40] * 8, p_bits=[60, 60], alpha=2, log_scale=40),
     dict(graph="er", V=40, deg=3.0, F=7, Fp=3, seed=5), 4, 2, True, "random"),
    (dict(log_n=12, q_bits=[60, 40, 40], p_bits=[60], alpha=1, log_scale=40),
     dict(graph="er", V=64, deg=4.0, F=16, Fp=8, seed=0), 4, 11, True, "random"),
    (dict(log_n=13, q_bits=[60] + [45] * 10, p_bits=[60] * 3, alpha=3, log_scale=45),
     dict(graph="chung_lu", V=2000, deg=4.5, gamma=2.5, F=9, Fp=16, x="tfidf", w="glorot", seed=7),
     1, 2, True, "random"),
]


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_library_planner_matches_oracle_planner(ci):
    prm, wk, t, radix, aoo, order = CASES[ci]
    P = ckks.Params(prm["log_n"], prm["q_bits"], prm["p_bits"], prm["alpha"], prm["log_scale"])
    w = wl.make_workload(**wk)
    B = P.slots // t
    perm = wl.identity_order(w.V) if order == "identity" else wl.random_order(w.V, B, ci)
    op = planner.build_plan(P, P.L, w.row_ptr, w.col, w.val, w.V, w.W, perm, t, radix, aoo)
    want = oracle_records(op)
    got = fg.plan_dry_run(prm, w.row_ptr, w.col, w.val, w.W, perm, t=t, radix_bits=radix, aoo=aoo)
    assert got.shape == want.shape
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("in_level,t", [(9, 1), (5, 4)])
def test_planner_from_a_lower_input_level(in_level, t):
    """A second layer starts below the top level (after the first layer and
    the x^2 activation): both planners take the input level."""
    prm = dict(log_n=11, q_bits=[60] + [40] * 12, p_bits=[60, 60], alpha=2, log_scale=40)
    P = ckks.Params(prm["log_n"], prm["q_bits"], prm["p_bits"], prm["alpha"], prm["log_scale"])
    w = wl.make_workload(graph="chung_lu", V=200, deg=4.0, gamma=2.5, F=16, Fp=3, seed=5)
    perm = wl.random_order(w.V, P.slots // t, 5)
    op = planner.build_plan(P, in_level, w.row_ptr, w.col, w.val, w.V, w.W, perm, t, 3, True)
    got = fg.plan_dry_run(prm, w.row_ptr, w.col, w.val, w.W, perm, t=t, radix_bits=3, in_level=in_level)
    np.testing.assert_array_equal(got, oracle_records(op))
    assert got[7] == in_level


def test_packing_rule_matches_oracle():
    prm = dict(log_n=12, q_bits=[60, 40, 40], p_bits=[60], alpha=1, log_scale=40)
    w = wl.config_workload("toy")
    P = ckks.Params(12, [60, 40, 40], [60], 1, 40)
    n = int(np.floor(w.mean_degree() + 0.5))
    t = planner.choose_t(w.X.shape[1], n, w.V, w.W.shape[1], P.slots)
    perm = wl.identity_order(w.V)
    got = fg.plan_dry_run(prm, w.row_ptr, w.col, w.val, w.W, perm, t=0, radix_bits=11)
    assert got[2] == t == 4


def test_auto_radix_fits_budget_and_errors():
    prm = dict(log_n=11, q_bits=[60] + [40] * 5, p_bits=[60], alpha=1, log_scale=40)
    w = wl.make_workload(graph="er", V=100, deg=4.0, F=3, Fp=2, seed=3)
    perm = wl.random_order(w.V, 1024, 3)
    rec = fg.plan_dry_run(prm, w.row_ptr, w.col, w.val, w.W, perm, t=1)
    n_groups, out_level = rec[11], rec[8]
    assert out_level >= 0 and n_groups <= 4
    with pytest.raises(fg.FicgcnError) as e:
        fg.plan_dry_run(prm, w.row_ptr, w.col, w.val, w.W, perm, t=1, radix_bits=1)
    assert e.value.code == -2   # FG_ELEVEL
    bad = perm.copy()
    bad[1] = bad[0]
    with pytest.raises(fg.FicgcnError) as e:
        fg.plan_dry_run(prm, w.row_ptr, w.col, w.val, w.W, bad, t=1)
    assert e.value.code == -1   # FG_EINVAL


def test_benchmark_plan_matches_oracle_and_merges():
    """The benchmark's own layer plan (power-law graph with hubs, 19,717 nodes,
    N = 2^16, radix 4): identical in both planners, and in-flight sums occur
    (masks other than the accumulator's carrying edge weights)."""
    c = wl.CONFIGS["pubmed_like"]
    P = ckks.Params(c["log_n"], c["q_bits"], c["p_bits"], c["alpha"], c["log_scale"])
    w = wl.config_workload("pubmed_like")
    perm = wl.random_order(w.V, P.slots, 2025)
    op = planner.build_plan(P, P.L, w.row_ptr, w.col, w.val, w.V, w.W, perm, 1, 2, True, 10)
    got = fg.plan_dry_run(c, w.row_ptr, w.col, w.val, w.W, perm, t=1, radix_bits=2, min_out_level=10)
    np.testing.assert_array_equal(got, oracle_records(op))
    weighted = sum(1 for g in op.groups for tm in g.terms
                   if tm.dst >= 0 and np.any((op.masks[tm.mask].values != 0) &
                                             (op.masks[tm.mask].values != 1)))
    assert weighted > 0
    assert max(g.n_out for g in op.groups) <= 32
