"""The encrypted layer A-hat X W, executed step by step.  TEST INFRASTRUCTURE ONLY.

Steps (paper Sec. 3.2-3.3, App. B.1; readings in planner.py):
  1. combination Z_j = sum_f W[f, j] X_f on the packed inputs:
     t = 1: integer constants c = round(W[f,j] * q_l) times each input
            ciphertext, summed, then one rescale by q_l;
     t > 1: block-replicated W plaintexts times each input, summed,
            rescaled, then rotate-and-sum ct <- ct + Rot(ct, B*2^i) for
            i = 0..log t - 1 so block 0 holds the whole sum;
  2. SpIntra-CA groups: per input lane one ModUp shared by all its
     rotations, every term mask (x) source added into its output lane or
     the accumulator, then every output rescaled; the running accumulator
     is dropped one limb and the group's arrivals added;
  3. the accumulator after the last group is the layer output.
"""
import numpy as np

from . import ckks
from .planner import ACC


def encode_plan_masks(params, plan):
    """Every mask of the plan encoded at scale q_level, level = its level."""
    return [ckks.encode(params, m.values, float(params.q[m.level]), m.level)
            for m in plan.masks]


def combination(params, plan, cts_in, keys, pts, column):
    """Z_j for one output column j (step 1)."""
    l0 = plan.in_level
    if plan.t == 1:
        acc = np.zeros((2, l0 + 1, params.n), dtype=np.uint64)
        for f in range(plan.F):
            ckks.const_mac(params, acc, cts_in[f], plan.comb_consts[f][column])
    else:
        acc = None
        for b in range(len(plan.comb_masks)):
            prod = ckks.pmult(params, pts[plan.comb_masks[b][column]], cts_in[b])
            acc = prod if acc is None else ckks.add_ct(params, acc, prod)
    z = ckks.rescale_ct(params, acc)
    for k in (plan.comb_rots or []):
        z = ckks.add_ct(params, z, ckks.rotate(params, z, k, keys[k % plan.M]))
    return z


def aggregation(params, plan, z, keys, pts):
    """SpIntra-CA on one column ciphertext z (step 2)."""
    lanes = [z]
    acc = None
    for grp in plan.groups:
        assert all(ckks.level_of(c) == grp.level for c in lanes)
        need = sorted({a for (a, _) in grp.rotations})
        digits = {a: ckks.modup(params, lanes[a][1], grp.level) for a in need}
        rot = {(a, k): ckks.rotate(params, lanes[a], k, keys[k % plan.M], digits[a])
               for (a, k) in grp.rotations}
        outs = [None] * grp.n_out
        acc_new = None
        for tm in grp.terms:
            src = lanes[tm.src] if tm.k == 0 else rot[(tm.src, tm.k)]
            prod = ckks.pmult(params, pts[tm.mask], src)
            if tm.dst == ACC:
                acc_new = prod if acc_new is None else ckks.add_ct(params, acc_new, prod)
            else:
                o = outs[tm.dst]
                outs[tm.dst] = prod if o is None else ckks.add_ct(params, o, prod)
        lanes = [ckks.rescale_ct(params, o) for o in outs]
        if acc is not None:
            acc = ckks.drop_ct(acc)
        if acc_new is not None:
            acc_new = ckks.rescale_ct(params, acc_new)
            acc = acc_new if acc is None else ckks.add_ct(params, acc, acc_new)
    return acc


def layer_axw(params, plan, cts_in, keys, pts, columns=None):
    """Output ciphertexts (one per output column) of the layer."""
    cols = range(plan.Fp) if columns is None else columns
    return [aggregation(params, plan, combination(params, plan, cts_in, keys, pts, j),
                        keys, pts) for j in cols]
