"""SpIntra-CA planner of the oracle.  TEST INFRASTRUCTURE ONLY.

Written from the paper's description of the method:
  * latency-aware packing (Sec. 3.2, App. B.1): J(t; F, n) = 2*ceil(F*n/t) +
    20*ceil(log t) when M > V*F'; t = 1 when M <= V*F';
  * column-major packing of t columns per ciphertext (App. B.1), blocks of
    B = M/t slots, node v of column f of block k at slot k*B + perm[v];
  * SpIntra-CA (Sec. 3.3): per-node rotation lengths, processed from the low
    bits upward, nodes whose step bit is 0 stay, moved and kept values are
    selected by 0/1 masks, a node that reaches its target is removed and
    added to the result ciphertext, and slot conflicts open extra
    ciphertexts;
  * AOO (Sec. 3.3.2): each shift is the shortest cyclic distance;
  * CPOO (Sec. 3.3.2): consecutive bit steps merged into one rotation (the
    radix-2^r groups below), and sparse ciphertexts merged (the first-fit
    lane assignment below).

Readings the paper leaves open (the library implements the same):
  * a "token" is one edge v <- u (u != v) of A-hat; the self term A[v,v] is
    multiplied in at group 0;
  * bits are taken r at a time (radix 2^r): group g handles bits
    [g*r, g*r + r) of |shift|; one rotation per distinct signed digit
    amount; one mask product and one rescale per group;
  * in-flight reduction: moving tokens that reach the same slot on the way
    to the same destination are summed from then on -- each multiplied by
    its edge weight in that step's mask -- and travel as one carrier with
    weight 1 (an extension of the paper's removal-on-arrival: the sum is
    formed earlier, so converging neighbours of a hub need no extra lanes);
  * assignment: unchanged tokens are grouped into items (one source slot and
    rotation, one new slot) visited in the order (source lane, rotation
    amount mod M, new slot), then the new carriers in the order (new slot,
    destination); an item joins the lowest output lane that already holds
    its content at that slot, else the lowest lane whose slot is free, else
    opens a new lane (the conflict);
  * every mask is encoded at scale q_l, l the level of the group, so the
    rescale that ends the group returns the ciphertext scale to Delta.

The plan is pure structure: which rotations, which masked products, and
each mask's slot values.  Encoding the masks is ckks.encode's job.
"""
import math
from dataclasses import dataclass, field

import numpy as np

ACC = -1  # destination "accumulator" in a term


def packing_objective(t, F, n):
    """J(t; F, n) = 2*ceil(F*n/t) + 20*ceil(log2 t)  (App. B.1)."""
    return 2 * (-(-F * n // t)) + 20 * math.ceil(math.log2(t)) if t > 1 else 2 * F * n


def choose_t(F, n, V, Fp, M):
    """Columns per ciphertext: t = 1 if M <= V*F'; otherwise the power of two
    t <= min(F, M/V) minimising J, ties to the smaller t."""
    if M <= V * Fp:
        return 1
    best_t, best_j = 1, packing_objective(1, F, n)
    t = 2
    while t <= F and t * V <= M:
        j = packing_objective(t, F, n)
        if j < best_j:
            best_t, best_j = t, j
        t *= 2
    return best_t


def shift_amount(src_slot, dst_slot, M, aoo=True):
    """Rotation amount rho with Rot(ct, rho) carrying slot src to slot dst
    (Rot(.,k) moves slot j+k to slot j): rho = src - dst mod M; with AOO the
    representative of least magnitude, in (-M/2, M/2]."""
    r = (src_slot - dst_slot) % M
    if aoo and r > M // 2:
        r -= M
    return r


@dataclass
class Term:
    src: int       # input lane
    k: int         # signed rotation amount, 0 = the lane itself
    dst: int       # output lane, or ACC
    mask: int      # index into Plan.masks


@dataclass
class Group:
    bit_lo: int
    n_bits: int
    level: int                 # level of the products; the rescale drops q_level
    n_in: int
    n_out: int
    rotations: list            # [(src lane, k)], k != 0
    terms: list                # [Term]


@dataclass
class Mask:
    level: int
    values: np.ndarray         # M slot values (float64)


@dataclass
class Plan:
    n: int
    M: int
    t: int
    B: int
    V: int
    F: int
    Fp: int
    perm: np.ndarray           # node -> slot in [0, B)
    in_level: int
    comb_consts: list = None   # t == 1: [F][F'] signed integers round(W*q_l)
    comb_masks: list = None    # t > 1: [ceil(F/t)][F'] mask indices
    comb_rots: list = None     # t > 1: rotation amounts B*2^i
    groups: list = field(default_factory=list)
    masks: list = field(default_factory=list)
    out_level: int = 0
    radix_bits: int = 0
    aoo: bool = True
    n_copies: int = 0          # Inter-CA: one mask per neighbour copy (masks 0..n_copies-1)

    def rotation_amounts(self):
        ks = set()
        for k in (self.comb_rots or []):
            ks.add(k % self.M)
        for g in self.groups:
            for (_, k) in g.rotations:
                ks.add(k % self.M)
        return sorted(ks)

    def rotation_count(self):
        return (len(self.comb_rots or []) * self.Fp
                + sum(len(g.rotations) for g in self.groups) * self.Fp)


def build_plan(params, in_level, row_ptr, col, val, V, W, perm, t,
               radix_bits, aoo=True, min_out_level=0):
    """Plan of one layer A-hat (X W) for ciphertexts at level in_level."""
    n, M = params.n, params.slots
    F, Fp = W.shape
    B = M // t
    perm = np.asarray(perm, dtype=np.int64)
    if perm.shape[0] != V or len(set(perm.tolist())) != V or perm.min() < 0 or perm.max() >= B:
        raise ValueError("perm must be an injection of the V nodes into [0, B)")
    plan = Plan(n=n, M=M, t=t, B=B, V=V, F=F, Fp=Fp, perm=perm, in_level=in_level,
                radix_bits=radix_bits, aoo=aoo)

    # --- combination (App. B.1): Z_j = sum_f W[f,j] X_f, scale kept at Delta
    ql = params.q[in_level]
    if t == 1:
        plan.comb_consts = [[int(_round_half_away(float(W[f, j]) * float(ql)))
                             for j in range(Fp)] for f in range(F)]
    else:
        nb = -(-F // t)
        plan.comb_masks = []
        for b in range(nb):
            row = []
            for j in range(Fp):
                vals = np.zeros(M)
                for kk in range(t):
                    f = b * t + kk
                    if f < F:
                        vals[kk * B:(kk + 1) * B] = W[f, j]
                plan.masks.append(Mask(level=in_level, values=vals))
                row.append(len(plan.masks) - 1)
            plan.comb_masks.append(row)
        plan.comb_rots = [B << i for i in range(int(math.log2(t)))]

    # --- tokens: one per edge v <- u, u != v
    self_w = np.zeros(V)
    toks = []   # [content, lane, pos, rho, dest, w]; content u >= 0 is node u's value
    for v in range(V):
        for e in range(row_ptr[v], row_ptr[v + 1]):
            u = int(col[e])
            w = float(val[e])
            if u == v:
                self_w[v] += w
            else:
                rho = shift_amount(int(perm[u]), int(perm[v]), M, aoo)
                toks.append([u, 0, int(perm[u]), rho, int(perm[v]), w])
    max_abs = max((abs(tk[3]) for tk in toks), default=0)
    total_bits = max_abs.bit_length()
    G = max(1, -(-total_bits // radix_bits))
    level = in_level - 1
    if level - G < min_out_level:
        raise ValueError("level budget exhausted: %d groups from level %d" % (G, level))

    n_lanes = 1
    n_carriers = 0
    for g in range(G):
        lo = g * radix_bits
        nb = max(0, min(radix_bits, total_bits - lo))
        gterms = {}      # (src lane, k, dst) -> {slot: mask value}
        if g == 0 and np.any(self_w != 0):
            gterms[(0, 0, ACC)] = {int(perm[v]): float(self_w[v]) for v in range(V) if self_w[v] != 0}
        # step of every token in this group
        rots = set()
        moving = []      # (token, k, new slot)
        for tk in toks:
            content, lane, pos, rho, dest, w = tk
            digit = (abs(rho) >> lo) & ((1 << nb) - 1) if nb > 0 else 0
            k = (digit << lo) * (1 if rho > 0 else -1)
            newpos = (pos - k) % M
            if k != 0:
                rots.add((lane, k))
            if rho - k == 0:                       # arrival: removed into the accumulator
                d = gterms.setdefault((lane, k, ACC), {})
                assert newpos == dest and dest not in d
                d[dest] = w
            else:
                moving.append((tk, k, newpos))
        # tokens meeting at one slot on the way to one destination are summed
        # from here on (each weighted by its own edge weight in this step's mask)
        by_pd = {}
        for m in moving:
            by_pd.setdefault((m[2], m[0][4]), []).append(m)
        items = {}       # (lane, k, new slot) -> tokens carried unchanged
        merged = []
        for (p, d), ms in by_pd.items():
            if len(ms) >= 2:
                merged.append((p, d, ms))
            else:
                tk, k, _ = ms[0]
                items.setdefault((tk[1], k, p), []).append(tk)
        out_slots = []   # per output lane: {slot: content}
        nxt = []

        def place(p, content):
            x = next((i for i, sl in enumerate(out_slots) if sl.get(p) == content), None)
            if x is not None:
                return x, True
            x = next((i for i, sl in enumerate(out_slots) if p not in sl), None)
            if x is None:
                out_slots.append({})
                x = len(out_slots) - 1
            out_slots[x][p] = content
            return x, False

        for key in sorted(items, key=lambda z: (z[0], z[1] % M, z[2])):
            lane, k, p = key
            tks = items[key]
            content = tks[0][0]
            assert all(t[0] == content for t in tks)
            x, joined = place(p, content)
            if not joined:
                gterms.setdefault((lane, k, x), {})[p] = 1.0
            for t in tks:
                nxt.append([content, x, p, t[3] - k, t[4], t[5]])
        for (p, d, ms) in sorted(merged, key=lambda z: (z[0], z[1])):
            n_carriers += 1
            content = -n_carriers
            x, joined = place(p, content)
            assert not joined
            for (tk, k, _) in ms:
                entry = gterms.setdefault((tk[1], k, x), {})
                assert p not in entry
                entry[p] = tk[5]
            rho2 = ms[0][0][3] - ms[0][1]
            assert all(t[3] - kk == rho2 for (t, kk, _) in ms)
            nxt.append([content, x, p, rho2, d, 1.0])
        # canonical order of the terms; masks numbered in that order
        terms = []
        for (src, k, dst) in sorted(gterms, key=lambda z: (z[0], z[1] % M, z[2])):
            vals = np.zeros(M)
            for sl, v in gterms[(src, k, dst)].items():
                vals[sl] = v
            plan.masks.append(Mask(level=level, values=vals))
            terms.append(Term(src, k, dst, len(plan.masks) - 1))
        plan.groups.append(Group(bit_lo=lo, n_bits=nb, level=level, n_in=n_lanes,
                                 n_out=len(out_slots),
                                 rotations=sorted(rots, key=lambda r: (r[0], r[1] % M)),
                                 terms=terms))
        toks = nxt
        n_lanes = len(out_slots)
        level -= 1
    assert not toks, "tokens left after the last group"
    plan.out_level = level
    return plan


def _round_half_away(x):
    """Nearest integer, ties away from zero (as C round()); exact for every double."""
    a = abs(x)
    f = math.floor(a)
    r = f + (1 if a - f >= 0.5 else 0)
    return r if x >= 0 else -r


# ----------------------------------------------------------------------
# FP64 simulation of a plan (rotate = np.roll, mask = elementwise)
# ----------------------------------------------------------------------

def simulate_aggregation(plan, z):
    """Run the SpIntra-CA part of the plan on a plain slot vector z (length M)."""
    lanes = [np.asarray(z, dtype=np.float64)]
    acc = np.zeros(plan.M)
    for grp in plan.groups:
        rot = {(a, k): np.roll(lanes[a], -k) for (a, k) in grp.rotations}
        outs = [np.zeros(plan.M) for _ in range(grp.n_out)]
        for tm in grp.terms:
            src = lanes[tm.src] if tm.k == 0 else rot[(tm.src, tm.k)]
            prod = plan.masks[tm.mask].values * src
            if tm.dst == ACC:
                acc = acc + prod
            else:
                outs[tm.dst] = outs[tm.dst] + prod
        lanes = outs
    return acc


def simulate_combination(plan, X, W):
    """Slot vectors Z_j after the combination, from the packed plain X."""
    V, F = X.shape
    M, B, t = plan.M, plan.B, plan.t
    nb = -(-F // t)
    packed = []
    for b in range(nb):
        v = np.zeros(M)
        for kk in range(t):
            f = b * t + kk
            if f < F:
                v[kk * B + plan.perm] = X[:, f]
        packed.append(v)
    Z = []
    for j in range(plan.Fp):
        if t == 1:
            z = sum(W[f, j] * packed[f] for f in range(F))
        else:
            z = sum(plan.masks[plan.comb_masks[b][j]].values * packed[b] for b in range(nb))
            for k in plan.comb_rots:
                z = z + np.roll(z, -k)
        Z.append(z)
    return Z


def build_inter_plan(params, in_level, nbr, wts, V, W, perm):
    """Inter-CA plan (Sec. 3.1, Table 1: aggregation by PMult and Add over n
    node arrangements the client encrypts).  Copy k of the input holds row
    nbr[v][k] of X at slot perm[v]; the layer computes Z_k = X_k W (the
    combination of App. B.1 on every copy, constants at q_l) and then
    sum_k mask_k (x) Z_k with mask_k holding wts[v][k] at perm[v] (scale
    q_{l-1}); two rescales.  The records mark it with radix_bits = -n."""
    M = params.slots
    F, Fp = W.shape
    nbr = np.asarray(nbr)
    n = nbr.shape[1]
    perm = np.asarray(perm, dtype=np.int64)
    if perm.shape[0] != V or len(set(perm.tolist())) != V or perm.min() < 0 or perm.max() >= M:
        raise ValueError("perm must be an injection of the V nodes into [0, M)")
    plan = Plan(n=params.n, M=M, t=1, B=M, V=V, F=F, Fp=Fp, perm=perm, in_level=in_level,
                radix_bits=-n, aoo=True, n_copies=n)
    ql = params.q[in_level]
    plan.comb_consts = [[int(_round_half_away(float(W[f, j]) * float(ql))) for j in range(Fp)]
                        for f in range(F)]
    for k in range(n):
        vals = np.zeros(M)
        for v in range(V):
            if nbr[v, k] >= 0:
                vals[perm[v]] = wts[v, k]
        plan.masks.append(Mask(level=in_level - 1, values=vals))
    plan.out_level = in_level - 2
    return plan


# ----------------------------------------------------------------------
# aggregation mode of a layer (Sec. 3.4 "Selecting Aggregation Mode",
# App. B.2, Table 1)
# ----------------------------------------------------------------------
SPINTRA, INTER = 0, 1


def mode_costs(F, t, n, R, T, lat=(20.0, 1.0, 1.0)):
    """Latency of one output column in each mode, from Table 1's operation
    counts: Inter-CA applies the combination to each of the n node
    arrangements (n ceil(F/t) PMult + Add), sums the n masked copies (n PMult
    + Add) and needs ceil(log2 t) Rot for the packing; SpIntra-CA applies the
    combination once (ceil(F/t) PMult + Add), the same ceil(log2 t) Rot, and
    its plan's R rotations and T masked terms (PMult + Add each).
    lat = (L_rot, L_pmult, L_add).  Returns (SpIntra-CA, Inter-CA)."""
    l_rot, l_pm, l_add = lat
    nb = -(-F // t)
    lg = math.ceil(math.log2(t)) if t > 1 else 0
    inter = (n * nb + n) * (l_pm + l_add) + lg * l_rot
    spintra = (nb + T) * (l_pm + l_add) + (lg + R) * l_rot
    return spintra, inter


def paper_mode_estimates(F, t, n, V, c=1.0):
    """The paper's estimates (Sec. 3.4): Inter-CA 2 ceil(F n / t), SpIntra-CA
    10 c n log^2 V (V nodes; c in [0, 1] left open by the paper)."""
    return 10.0 * c * n * math.log2(V) ** 2, 2 * (-(-F * n // t))


def select_mode(plan, layer, n_copies, lat=(20.0, 1.0, 1.0), max_inter_cts=0):
    """Mode of one layer given its SpIntra-CA plan: the first layer (0) is
    Inter-CA, whose copies the client encrypts offline, unless its input
    (n ceil(F/t) ciphertexts) exceeds max_inter_cts (0: no limit); a later
    layer takes the cheaper mode of mode_costs, ties to SpIntra-CA.  The
    plan's exact counts R, T stand in for the paper's 10 c n log^2 V.
    Returns (mode, (SpIntra-CA cost, Inter-CA cost), (R, T))."""
    R = sum(len(g.rotations) for g in plan.groups)
    T = sum(len(g.terms) for g in plan.groups)
    costs = mode_costs(plan.F, plan.t, n_copies, R, T, lat)
    fits = max_inter_cts <= 0 or n_copies * (-(-plan.F // plan.t)) <= max_inter_cts
    if layer == 0:
        mode = INTER if fits else SPINTRA
    else:
        mode = INTER if (fits and costs[1] < costs[0]) else SPINTRA
    return mode, costs, (R, T)
