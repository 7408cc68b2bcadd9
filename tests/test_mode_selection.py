"""Aggregation-mode selection (paper Sec. 3.4 "Selecting Aggregation Mode",
App. B.2, Table 1) in both planners: hand-worked cases and the library's
host planner against the oracle's."""
import numpy as np
import pytest

from oracle import ckks, planner
from paper_2506_10399_gb300 import workloads as wl

PRM = dict(log_n=10, q_bits=[60] + [40] * 6, p_bits=[60, 60], alpha=2, log_scale=40)
P = ckks.Params(PRM["log_n"], PRM["q_bits"], PRM["p_bits"], PRM["alpha"], PRM["log_scale"])


def two_nodes(F):
    """Nodes u = 0, v = 1 joined by one edge, at slots 0 and 1: every entry
    of A-hat = D^-1/2 (A + I) D^-1/2 is 1/2, each row has n = 2 entries."""
    row_ptr = np.array([0, 2, 4])
    col = np.array([0, 1, 0, 1])
    val = np.full(4, 0.5)
    W = np.ones((F, 2)) / F
    perm = np.array([0, 1])
    return row_ptr, col, val, W, perm


@pytest.mark.parametrize("F,layer,lat,cap,want", [
    # One radix-2 group: the self term, and the two neighbours arriving by
    # Rot(-1) and Rot(+1) -> R = 2 rotations, T = 3 masked terms.  With
    # t = 1, n = 2 and (L_rot, L_pmult, L_add) = (20, 1, 1):
    #   SpIntra-CA = (F + 3) 2 + 2 * 20,   Inter-CA = (2F + 2) 2,
    # so Inter-CA is cheaper exactly when F < 21 (F = 21 ties: SpIntra-CA).
    (20, 1, (20.0, 1.0, 1.0), 0, planner.INTER),       # 84 < 86
    (21, 1, (20.0, 1.0, 1.0), 0, planner.SPINTRA),     # 88 = 88
    (64, 1, (20.0, 1.0, 1.0), 0, planner.SPINTRA),     # 260 > 174
    # measured-style latencies (5, 1, 0.5), F = 8: SpIntra-CA 11 * 1.5 + 2 * 5
    # = 26.5 against Inter-CA 18 * 1.5 = 27
    (8, 1, (5.0, 1.0, 0.5), 0, planner.SPINTRA),
    # the first layer is Inter-CA whatever the costs (the client's copies)...
    (64, 0, (20.0, 1.0, 1.0), 0, planner.INTER),
    # ... unless its 2 * 64 input ciphertexts exceed the client's budget
    (64, 0, (20.0, 1.0, 1.0), 100, planner.SPINTRA),
])
def test_hand_worked_selection(F, layer, lat, cap, want):
    row_ptr, col, val, W, perm = two_nodes(F)
    plan = planner.build_plan(P, P.L, row_ptr, col, val, 2, W, perm, 1, 1)
    mode, costs, (R, T) = planner.select_mode(plan, layer, 2, lat, cap)
    assert (R, T) == (2, 3)
    lr, lp, la = lat
    assert costs == pytest.approx(((F + 3) * (lp + la) + 2 * lr, (2 * F + 2) * (lp + la)))
    assert mode == want


def test_paper_estimates():
    """Sec. 3.4's formulas: Inter-CA 2 ceil(F n / t), SpIntra-CA 10 c n log^2 V."""
    sp, inter = planner.paper_mode_estimates(F=100, t=4, n=5, V=1024, c=0.5)
    assert inter == 2 * 125 and sp == pytest.approx(10 * 0.5 * 5 * 100)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("layer,cap", [(0, 0), (1, 0), (1, 50)])
def test_library_selection_matches_oracle(seed, layer, cap):
    fg = pytest.importorskip("paper_2506_10399_gb300")
    w = wl.make_workload(graph="chung_lu", V=40 + 20 * seed, deg=3.0 + seed, gamma=2.5, F=6 + 5 * seed,
                         Fp=3, seed=seed)
    perm = wl.random_order(w.V, P.slots, seed)
    n = w.max_degree()
    lat = (10.0 + seed, 1.0, 0.25 * (seed + 1))
    op = planner.build_plan(P, P.L, w.row_ptr, w.col, w.val, w.V, w.W, perm, 1, 3)
    want_mode, want_costs, (R, T) = planner.select_mode(op, layer, n, lat, cap)
    mode, costs, cnt = fg.select_mode(PRM, w.row_ptr, w.col, w.val, w.W, perm, layer, n, lat, cap,
                                      t=1, radix_bits=3)
    assert mode == want_mode
    assert (cnt["rotations"], cnt["terms"]) == (R, T)
    assert cnt["inter_inputs"] == n * w.X.shape[1]
    assert (costs["spintra"], costs["inter"]) == pytest.approx(want_costs)
