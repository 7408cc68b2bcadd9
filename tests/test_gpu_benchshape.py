"""The layer at the benchmark's kernel shapes, word for word against the
oracle's stored output (tests/golden/benchshape_layer.json, written by
tests/golden/make_benchshape_layer.py from oracle/ alone).

Shapes reached (the launch configuration bench.py times on pubmed_like):
N = 2^16 with 20 + 4 primes, 5 key-switching digits at level 18 (k_ks_ip<5>
with P phi(c0) folded in), 16 output columns (32 polynomials: two polynomial
groups per group-MAC tile), groups of up to 11 outputs (three thread groups
per CTA) and up to 47 sources (split over two launches), the fused ModDown +
rescale at 23 extended limbs, and a 136-column combination (two 128-column
chunks; from host memory also three 64-column copy chunks).  The inputs are
integer-defined (uniform residues, integer masks), so the stored digests hold
on any platform."""
import hashlib
import json
import os

import numpy as np
import pytest

from oracle import ckks, planner
from paper_2506_10399_gb300 import workloads as wl
from plan_records import oracle_records

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "benchshape_layer.json")


def digest(ct):
    return hashlib.sha256(np.ascontiguousarray(ct, dtype="<u8").tobytes()).hexdigest()


@pytest.fixture(scope="module")
def case():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    fg = __graft_entry__.build()
    doc = json.load(open(GOLDEN))
    R = doc["recipe"]
    cfg = wl.CONFIGS[R["config"]]
    ctx = fg.Context(**cfg)
    P = ckks.Params(cfg["log_n"], cfg["q_bits"], cfg["p_bits"], cfg["alpha"], cfg["log_scale"])
    w = wl.make_workload(**R["graph"])
    perm = wl.random_order(w.V, R["window"], R["order_seed"])
    op = planner.build_plan(P, P.L, w.row_ptr, w.col, w.val, w.V, w.W, perm, R["t"],
                            R["radix_bits"], min_out_level=R["min_out_level"])
    plan = fg.plan_build(ctx, w.row_ptr, w.col, w.val, w.W, perm, t=R["t"],
                         radix_bits=R["radix_bits"], min_out_level=R["min_out_level"])
    np.testing.assert_array_equal(plan.describe(), oracle_records(op))
    for i, m in enumerate(op.masks):
        ints = wl.random_small_poly(P.n, R["mask_bits"], R["mask_seed"] + i)
        plan.set_plaintext(i, np.stack([np.mod(ints, np.int64(q)).astype(np.uint64)
                                        for q in P.q[:m.level + 1]]))
    sk, evk = fg.keygen(ctx, R["key_seed"], plan.rotation_amounts())
    keys = fg.load_evk(ctx, evk)
    del evk
    F = w.X.shape[1]
    x = np.empty((F, 2, P.L + 1, P.n), np.uint64)
    for f in range(F):
        for part in range(2):
            x[f, part] = wl.random_words(P.q, P.n, R["input_seed"] + 2 * f + part)
    return fg, ctx, doc, op, plan, keys, x


def test_benchshape_plan_reaches_the_benchmark_kernel_shapes(case):
    fg, ctx, doc, op, plan, keys, x = case
    shapes = doc["groups"]
    assert op.groups[0].level == 18 and -(-(18 + 1) // 4) == 5      # five digits
    assert max(g["n_out"] for g in shapes) >= 7                     # three thread groups
    assert max(g["sources"] for g in shapes) > 36                   # split launches
    assert op.Fp == 16 and op.F > 128


@pytest.mark.parametrize("where,tuning", [("device", {}), ("host", {}),
                                          ("device", dict(ntt_cols=16, ntt_rows=16, modup_fused=0, gmac_regs=0)),
                                          ("device", dict(modup_fused=1, moddown_fused=1)),
                                          ("device", dict(ks_split=2)),
                                          ("device", dict(kara=0)),
                                          ("host", dict(kara=0, ks_split=1, gmac_regs=1)),
                                          ("device", dict(ntt_cols=8, ntt_rows=8, ntt_tw=1, ks_split=1,
                                                          ks_cols=2, modup_fused=1, moddown_fused=1,
                                                          gmac_groups=4, gmac_regs=1))])
def test_benchshape_layer_word_for_word(case, where, tuning):
    """Also under other launch configurations (the fused ModUp, the other
    NTT tiles and twiddle form, the other key-switch and group-MAC choices,
    the group MAC's products with four multiplies instead of Karatsuba's three)."""
    import torch
    fg, ctx, doc, op, plan, keys, x = case
    if where == "device":
        xin = torch.from_numpy(x.view(np.int64)).cuda()
    else:
        xin = x
    fg.set_tuning(ctx, **tuning)
    try:
        out, lvl, _ = fg.gcn_layer_axw(ctx, keys, plan, xin)
    finally:
        fg.set_tuning(ctx)
    assert lvl == doc["out_level"] == op.out_level
    for j, want in doc["columns"].items():
        o = out[int(j)]
        o = o.cpu().numpy().view(np.uint64) if hasattr(o, "cpu") else np.asarray(o)
        assert list(o.shape) == want["shape"]
        bad = [(p, l, i, v, int(o[p, l, i])) for p, l, i, v in want["samples"] if int(o[p, l, i]) != v]
        assert not bad, "column %s differs from the oracle at sampled words %s" % (j, bad[:4])
        assert digest(o) == want["sha256"], "column %s differs from the oracle" % j
