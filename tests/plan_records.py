"""The oracle planner's plan written as the library's plan records (the
record layout of fg_plan_describe), so the two planners can be compared
element by element.  Test helper: reads oracle objects only."""
import numpy as np


def oracle_records(plan):
    r = [plan.n, plan.M, plan.t, plan.B, plan.V, plan.F, plan.Fp, plan.in_level, plan.out_level,
         plan.radix_bits, 1 if plan.aoo else 0, len(plan.groups), len(plan.masks)]
    r += [int(v) for v in plan.perm]
    if plan.t == 1:
        r += [c for row in plan.comb_consts for c in row]
    else:
        r += [m for row in plan.comb_masks for m in row]
        r += [len(plan.comb_rots)] + list(plan.comb_rots)
    for g in plan.groups:
        r += [g.bit_lo, g.n_bits, g.level, g.n_in, g.n_out, len(g.rotations)]
        for (a, k) in g.rotations:
            r += [a, k]
        r += [len(g.terms)]
        for tm in g.terms:
            r += [tm.src, tm.k, tm.dst, tm.mask]
    for m in plan.masks:
        nz = np.nonzero(m.values)[0]
        r += [m.level, len(nz)]
        for s in nz:
            r += [int(s), int(np.float64(m.values[s]).view(np.int64))]
    return np.array(r, dtype=np.int64)
