"""The encrypted layer A-hat X W, executed step by step.  TEST INFRASTRUCTURE ONLY.

Steps (paper Sec. 3.2-3.3, App. B.1; readings in planner.py):
  1. combination Z_j = sum_f W[f, j] X_f on the packed inputs:
     t = 1: integer constants c = round(W[f,j] * q_l) times each input
            ciphertext, summed, then one rescale by q_l;
     t > 1: block-replicated W plaintexts times each input, summed,
            rescaled, then rotate-and-sum ct <- ct + Rot(ct, B*2^i) for
            i = 0..log t - 1 so block 0 holds the whole sum;
  2. SpIntra-CA groups, evaluated two ways:
     plain (group_step_plain): the paper's update {ct} <- {ct} (x) Mask1 (+)
       Rot({ct}, 2^(m-1)) (x) Mask2 (Sec. 3.3) as written: every rotation is
       a complete Rot(c, k) with its own ModDown, every term a PMult of the
       mask and that ciphertext over q_0..q_l, the terms of an output added;
     double hoisted (group_step_double_hoisted, what the library computes):
       per input lane one ModUp shared by all its rotations; every output
       (lane or accumulator) is the sum of its terms Mask (x) source, where a
       rotated source Rot(c, k) = ModDown(u) + (phi_g(c0), 0) contributes
       Mask (x) phi_g(c0) directly and Mask (x) u to an extended-basis sum
       that is key-switched down with ONE ModDown per output (Bossuat et al.,
       Eurocrypt 2021); kept values contribute Mask (x) lane.
     The two differ by the ModDown rounding only: with C(x) the centred fast
     base conversion of x's special-prime residues, the double-hoisted output
     minus the plain one is exactly (sum_t m_t C(u_t) - C(sum_t m_t u_t)) / P
     (tests/test_oracle_layer.py pins this on big integers).  Then every
     output is rescaled, and the running accumulator is dropped one limb and
     receives the group's arrivals;
  3. the accumulator after the last group is the layer output.
"""
import numpy as np

from . import ckks
from .planner import ACC


def encode_plan_masks(params, plan):
    """Every mask of the plan encoded at scale q_level, level = its level,
    with residues over q_0..q_level and the special primes ([level+1+K][N])."""
    return [ckks.encode(params, m.values, float(params.q[m.level]), m.level, extended=True)
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


def _map(pool, fn, items):
    """fn over items, in a thread pool when one is given (the oracle's C core
    releases the interpreter lock); the results come back in item order."""
    items = list(items)
    return list(pool.map(fn, items)) if pool is not None else [fn(x) for x in items]


def group_step_double_hoisted(params, plan, grp, lanes, keys, pts, pool=None):
    """One SpIntra-CA group in the double-hoisted form: the outputs before
    their rescale ({dst: ct at grp.level}) and the extended-basis sums
    ({dst: [2][l+1+K][N]}) that were key-switched down.  pool: optional
    executor for the independent key switches and term products (sums are
    taken in term order either way)."""
    lv = grp.level
    assert all(ckks.level_of(c) == lv for c in lanes)
    qs = params.q[:lv + 1]
    ext_primes = params.ext_primes(lv)
    need = sorted({a for (a, _) in grp.rotations})
    digits = dict(zip(need, _map(pool, lambda a: ckks.modup(params, lanes[a][1], lv), need)))
    ks = dict(zip(grp.rotations, _map(
        pool, lambda r: ckks.keyswitch_ext(params, lanes[r[0]], r[1], keys[r[1] % plan.M], digits[r[0]]),
        grp.rotations)))
    ext = {}    # output -> extended-basis sum of Mask (x) u
    norm = {}   # output -> sum of Mask (x) phi_g(c0) and Mask (x) kept lane

    def add_into(d, key, val, primes):
        d[key] = val if key not in d else np.stack(
            [ckks.add_res(d[key][0], val[0], primes), ckks.add_res(d[key][1], val[1], primes)])

    def products(tm):
        m = pts[tm.mask]
        if tm.k == 0:
            return ckks.pmult(params, m[:lv + 1], lanes[tm.src]), None
        u, c0g = ks[(tm.src, tm.k)]
        prod = np.stack([ckks.poly_mul(params, m, u[0], ext_primes),
                         ckks.poly_mul(params, m, u[1], ext_primes)])
        c0part = np.stack([ckks.poly_mul(params, m[:lv + 1], c0g, qs),
                           np.zeros((lv + 1, params.n), dtype=np.uint64)])
        return c0part, prod

    for tm, (qpart, extpart) in zip(grp.terms, _map(pool, products, grp.terms)):
        add_into(norm, tm.dst, qpart, qs)
        if extpart is not None:
            add_into(ext, tm.dst, extpart, ext_primes)
    outs = {}
    for dst in set(ext) | set(norm):
        o = ckks.moddown_ct(params, ext[dst]) if dst in ext else None
        if dst in norm:
            o = norm[dst] if o is None else ckks.add_ct(params, o, norm[dst])
        outs[dst] = o
    return outs, ext


def group_step_plain(params, plan, grp, lanes, keys, pts):
    """One SpIntra-CA group in the paper's step order (Sec. 3.3): every
    rotation Rot(c, k) complete, with its own ModDown (ckks.rotate), then
    out[dst] = sum over its terms of PMult(mask, source) over q_0..q_l.
    The lifted digits of a lane are computed once and passed to each of its
    rotations: ModUp of the same c1 is the same whichever rotation asks, so
    this is the rotation of Sec. 2.1 in the hoisted order of reading R3.
    Returns the outputs before their rescale ({dst: ct at grp.level})."""
    lv = grp.level
    assert all(ckks.level_of(c) == lv for c in lanes)
    need = sorted({a for (a, _) in grp.rotations})
    digits = {a: ckks.modup(params, lanes[a][1], lv) for a in need}
    rot = {(a, k): ckks.rotate(params, lanes[a], k, keys[k % plan.M], digits[a])
           for (a, k) in grp.rotations}
    outs = {}
    for tm in grp.terms:
        src = lanes[tm.src] if tm.k == 0 else rot[(tm.src, tm.k)]
        prod = ckks.pmult(params, pts[tm.mask][:lv + 1], src)
        outs[tm.dst] = prod if tm.dst not in outs else ckks.add_ct(params, outs[tm.dst], prod)
    return outs


def close_group(params, grp, outs, acc):
    """Rescale every output of a group; the running accumulator (if any) is
    dropped one limb and receives the group's arrivals.  Returns the next
    lanes and the accumulator."""
    lanes = [ckks.rescale_ct(params, outs[x]) for x in range(grp.n_out)]
    if acc is not None:
        acc = ckks.drop_ct(acc)
    if ACC in outs:
        acc_new = ckks.rescale_ct(params, outs[ACC])
        acc = acc_new if acc is None else ckks.add_ct(params, acc, acc_new)
    return lanes, acc


def aggregation(params, plan, z, keys, pts, plain=False, pool=None):
    """SpIntra-CA on one column ciphertext z (step 2), double hoisted (the
    library's form) or, with plain set, in the paper's step order."""
    lanes = [z]
    acc = None
    for grp in plan.groups:
        if plain:
            outs = group_step_plain(params, plan, grp, lanes, keys, pts)
        else:
            outs, _ = group_step_double_hoisted(params, plan, grp, lanes, keys, pts, pool)
        lanes, acc = close_group(params, grp, outs, acc)
    return acc


def layer_axw(params, plan, cts_in, keys, pts, columns=None, plain=False, pool=None):
    """Output ciphertexts (one per output column) of the layer; plain selects
    the paper's step order for the SpIntra-CA groups (see aggregation), pool
    an optional thread pool for the double-hoisted form."""
    cols = range(plan.Fp) if columns is None else columns
    return [aggregation(params, plan, combination(params, plan, cts_in, keys, pts, j),
                        keys, pts, plain=plain, pool=pool) for j in cols]


def inter_ca_layer(params, plan, copies, pts, columns=None):
    """Inter-CA layer: for each output column j,
    Rescale(sum_k mask_k (x) Rescale(sum_f c_{f,j} X_{k,f})), the copies
    given copy-major (copies[k * F + f])."""
    cols = range(plan.Fp) if columns is None else columns
    F = plan.F
    out = []
    for j in cols:
        acc = None
        for k in range(plan.n_copies):
            z = combination(params, plan, copies[k * F:(k + 1) * F], None, pts, j)
            prod = ckks.pmult(params, pts[k], z)
            acc = prod if acc is None else np.stack(
                [ckks.add_res(acc[p], prod[p], params.q[:prod.shape[1]]) for p in range(2)])
        out.append(ckks.rescale_ct(params, acc))
    return out
