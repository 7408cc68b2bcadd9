"""bench.py's count of the contraction kernels' 32 x 32-bit products (its
ALU roof), read from the library's plan records, against the same counts
taken from the oracle's plan of the same graph:
  group MAC: terms x 2F' x N x (3 per limb below 2^46 in Karatsuba's form,
             else 4, over the group's l+1 limbs and the K special limbs);
  key switch: rotations x F' x E x N x 2 parts x beta digits x 4;
  combination: F x F' x 2 parts x (L+1) limbs x N x 4.
Host only: the records come from the library's planner without a device."""
import os
import sys

import pytest

from oracle import ckks, planner
from paper_2506_10399_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PARAMS = dict(log_n=12, q_bits=[60] + [45] * 5, p_bits=[60] * 2, alpha=2, log_scale=45)


class _Fg:
    @staticmethod
    def int_mul_peak(ctx, op):
        return 1e13


class _Ctx:
    def __init__(self, P):
        self.n, self.np, self.q = P.n, len(P.p), list(P.q)


class _Plan:
    def __init__(self, rec):
        self.rec = rec

    def describe(self):
        return self.rec


@pytest.mark.parametrize("kara", [0, 1])
def test_alu_product_counts_match_the_oracle_plan(kara):
    import __graft_entry__
    fg = __graft_entry__.build()
    sys.path.insert(0, ROOT)
    import bench
    P = ckks.Params(PARAMS["log_n"], PARAMS["q_bits"], PARAMS["p_bits"], PARAMS["alpha"], PARAMS["log_scale"])
    w = wl.make_workload(graph="chung_lu", V=300, deg=4.0, gamma=2.5, F=20, Fp=3, x="tfidf", w="glorot", seed=5)
    perm = wl.random_order(w.V, P.slots, 6)
    rec = fg.plan_dry_run(PARAMS, w.row_ptr, w.col, w.val, w.W, perm, t=1, radix_bits=3)
    op = planner.build_plan(P, P.L, w.row_ptr, w.col, w.val, w.V, w.W, perm, 1, 3)
    F, Fp, N, K = w.X.shape[1], w.W.shape[1], P.n, len(P.p)
    want_gm = want_ks = 0
    for g in op.groups:
        per_limb = sum(3 if (kara and q < (1 << 46)) else 4 for q in P.q[:g.level + 1]) + 4 * K
        want_gm += len(g.terms) * 2 * Fp * N * per_limb
        E = g.level + 1 + K
        beta = -(-(g.level + 1) // PARAMS["alpha"])
        want_ks += len(g.rotations) * Fp * E * N * 2 * beta * 4
    want_comb = F * Fp * 2 * (P.L + 1) * N * 4
    br = {k: {"ms": 1.0} for k in ("group_mac", "ks_ip", "comb")}
    out = bench.alu_roofline(_Fg(), _Ctx(P), _Plan(rec), br, F, Fp, PARAMS["alpha"], kara=kara)
    got = {k: v["mults"] for k, v in out["kernels"].items()}
    assert got["group_mac"] == want_gm
    assert got["ks_ip"] == want_ks
    assert got["comb"] == want_comb
    assert out["kernels"]["group_mac"]["achieved"] == want_gm / 1e-3


def test_traffic_ratio_only_for_the_profiled_sources(monkeypatch):
    """roofline.traffic: the committed ratio of ncu DRAM bytes to algorithmic
    bytes times this workload's algorithmic bytes, and null once the kernel
    sources (or the launch defaults) differ from those that were profiled."""
    sys.path.insert(0, ROOT)
    import json
    import bench
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        t = json.load(f)
    if t["sources_sha256"] != bench.sources_sha256():
        assert bench.traffic_for("group_mac", 1e9) is None
        pytest.skip("the kernel sources changed since profiles/ncu_traffic.json was captured")
    r = t["dram_over_algorithmic"]["group_mac"]
    assert bench.traffic_for("group_mac", 1e9) == pytest.approx(r * 1e9)
    assert bench.traffic_for("no_such_class", 1e9) is None
    monkeypatch.setattr(bench, "sources_sha256", lambda: "0" * 64)
    assert bench.traffic_for("group_mac", 1e9) is None
