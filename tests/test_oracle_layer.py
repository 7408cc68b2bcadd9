"""The oracle's layer evaluators pinned on the CPU.

* Double hoisting (reading R4) against the paper's step order (Sec. 3.3:
  every Rot complete with its own ModDown, then PMult, then Add): at every
  group of a multi-group layer, both forms start from the same lanes, and
  their outputs must differ by exactly
      D = (sum_t m_t * C(u_t) - C(sum_t m_t * u_t)) / P,
  with m_t the mask integers, u_t the key-switch outputs of the output's
  rotated terms, and C the centred fast base conversion of a polynomial's
  special-prime residues (y_k in (-p_k/2, p_k/2]).  D is computed here from
  its definition on Python integers (CRT lifts, schoolbook negacyclic
  products), and its size is bounded by (K/2) (sum_t ||m_t||_1 + 1).
* T2 (decryption within 2^-20 of FP64) for both evaluators, for the packed
  combination (t = 2, 4) and for the Inter-CA layer with its plan.
* Planted slips in either evaluator fail these pins.
"""
import numpy as np
import pytest

from oracle import ckks, layer, planner
from oracle.planner import ACC
from paper_2506_10399_gb300 import workloads as wl

BOUND = 2.0 ** -20


def lift(res, primes):
    """CRT lift of residues [len(primes)][N] to Python ints, centred."""
    M = 1
    for q in primes:
        M *= q
    acc = np.zeros(res.shape[1], dtype=object)
    for i, q in enumerate(primes):
        hat = M // q
        acc = acc + res[i].astype(object) * (hat * pow(hat % q, -1, q))
    acc = acc % M
    return np.where(acc > M // 2, acc - M, acc)


def centred_conversion(res_p, ps):
    """C(x) = sum_k y_k P/p_k, y_k = [x_k (P/p_k)^-1]_{p_k} in (-p_k/2, p_k/2]."""
    P = 1
    for p in ps:
        P *= p
    C = np.zeros(res_p.shape[1], dtype=object)
    for k, p in enumerate(ps):
        hat = P // p
        y = (res_p[k].astype(object) * pow(hat % p, -1, p)) % p
        y = np.where(y > p // 2, y - p, y)
        C = C + y * hat
    return C, P


def negacyclic_int(a, b):
    n = a.shape[0]
    full = np.convolve(a, b)
    out = full[:n].copy()
    out[:n - 1] -= full[n:]
    return out


def small_layer(t=1, radix=3, seed=8, V=24, F=6, Fp=2, log_n=10):
    P = ckks.Params(log_n, [60] + [40] * 6, [60, 60], 2, 40)
    w = wl.make_workload(graph="er", V=V, deg=3.0, F=F, Fp=Fp, seed=seed)
    perm = wl.random_order(w.V, P.slots // t, seed)
    plan = planner.build_plan(P, P.L, w.row_ptr, w.col, w.val, w.V, w.W, perm, t, radix)
    s = ckks.keygen_secret(P, seed)
    keys = {k: ckks.keygen_rotation(P, seed, s, k) for k in plan.rotation_amounts()}
    nb = -(-F // t)
    cts = []
    for b in range(nb):
        v = np.zeros(P.slots)
        for kk in range(t):
            f = b * t + kk
            if f < F:
                v[kk * plan.B + perm] = w.X[:, f]
        cts.append(ckks.encrypt(P, seed, b, ckks.encode(P, v, P.scale, P.L), s, P.L))
    pts = layer.encode_plan_masks(P, plan)
    return P, w, perm, plan, s, keys, cts, pts


@pytest.fixture(scope="module")
def case():
    return small_layer()


def moddown_difference(P, plan, grp, lanes, keys, pts, ext, dst):
    """D of the module docstring for one output, both parts, and its bound."""
    lv = grp.level
    ext_primes = P.ext_primes(lv)
    D = []
    bound = 0
    for part in range(2):
        Cs, Pp = centred_conversion(ext[dst][part][lv + 1:], P.p)
        acc = -Cs
        l1 = 0
        for tm in grp.terms:
            if tm.dst != dst or tm.k == 0:
                continue
            u, _ = ckks.keyswitch_ext(P, lanes[tm.src], tm.k, keys[tm.k % plan.M])
            Ct, _ = centred_conversion(u[part][lv + 1:], P.p)
            m = lift(pts[tm.mask], ext_primes)
            acc = acc + negacyclic_int(m, Ct)
            l1 += int(np.sum(np.abs(m)))
        assert all(int(v) % Pp == 0 for v in acc), "D is not an exact multiple of P"
        D.append(acc // Pp)
        bound = (P.K * (l1 + 1)) // 2 + 1
    return D, bound


def check_group_identity(P, plan, grp, lanes, keys, pts):
    dh, ext = layer.group_step_double_hoisted(P, plan, grp, lanes, keys, pts)
    pl = layer.group_step_plain(P, plan, grp, lanes, keys, pts)
    assert set(dh) == set(pl)
    qs = P.q[:grp.level + 1]
    for dst in dh:
        if dst not in ext:      # kept values only: no ModDown on either side
            np.testing.assert_array_equal(dh[dst], pl[dst])
            continue
        D, bound = moddown_difference(P, plan, grp, lanes, keys, pts, ext, dst)
        for part in range(2):
            diff = lift(ckks.sub_res(dh[dst][part], pl[dst][part], qs), qs)
            np.testing.assert_array_equal(diff, D[part])
            assert max(abs(int(v)) for v in D[part]) <= bound
    return dh, pl


def test_double_hoisting_equals_plain_up_to_the_moddown_term(case):
    """Every group of a three-group layer, started from the plain path's
    lanes: double-hoisted minus plain outputs == D exactly, |D| bounded."""
    P, w, perm, plan, s, keys, cts, pts = case
    assert len(plan.groups) >= 3
    z = layer.combination(P, plan, cts, keys, pts, 0)
    lanes, acc = [z], None
    for grp in plan.groups:
        _, pl = check_group_identity(P, plan, grp, lanes, keys, pts)
        lanes, acc = layer.close_group(P, grp, pl, acc)


@pytest.mark.parametrize("plain", [False, True])
def test_both_evaluators_decrypt_to_fp64(case, plain):
    P, w, perm, plan, s, keys, cts, pts = case
    outs = layer.layer_axw(P, plan, cts, keys, pts, plain=plain)
    ref = w.reference_output()
    for j, o in enumerate(outs):
        assert ckks.level_of(o) == plan.out_level
        d = ckks.decode(P, ckks.decrypt(P, o, s), P.scale).real
        assert np.max(np.abs(d[perm] - ref[:, j])) < BOUND


@pytest.mark.parametrize("t", [2, 4])
def test_packed_combination_layer_decrypts_to_fp64(t):
    """The t > 1 branch of the combination (App. B.1: block-replicated W
    plaintexts, then log t rotate-and-sum steps) through the whole layer."""
    P, w, perm, plan, s, keys, cts, pts = small_layer(t=t, seed=3, F=8, Fp=2)
    assert plan.t == t and len(plan.comb_rots) == int(np.log2(t))
    outs = layer.layer_axw(P, plan, cts, keys, pts)
    ref = w.reference_output()
    for j, o in enumerate(outs):
        d = ckks.decode(P, ckks.decrypt(P, o, s), P.scale).real
        assert np.max(np.abs(d[perm] - ref[:, j])) < BOUND


def inter_case(n=3, seed=6):
    P = ckks.Params(10, [60, 40, 40], [60], 1, 40)
    w = wl.make_workload(graph="er", V=20, deg=3.0, F=5, Fp=2, seed=seed)
    perm = wl.random_order(w.V, P.slots, seed)
    nbr, wts = wl.sample_neighbors(w, n, seed)
    plan = planner.build_inter_plan(P, P.L, nbr, wts, w.V, w.W, perm)
    s = ckks.keygen_secret(P, seed)
    copies = []
    for k in range(nbr.shape[1]):
        Xk = np.where((nbr[:, k] >= 0)[:, None], w.X[np.maximum(nbr[:, k], 0)], 0.0)
        for f in range(w.X.shape[1]):
            v = np.zeros(P.slots)
            v[perm] = Xk[:, f]
            copies.append(ckks.encrypt(P, seed + k, f, ckks.encode(P, v, P.scale, P.L), s, P.L))
    pts = layer.encode_plan_masks(P, plan)
    return P, w, perm, nbr, wts, plan, s, copies, pts


def test_inter_ca_layer_decrypts_to_the_sampled_product():
    """Inter-CA (Sec. 3.1, Table 1: PMult and Add over the client's node
    arrangements): build_inter_plan + inter_ca_layer decrypt within 2^-20 of
    FP64 sum_k w_k X[nbr_k] W, with no rotation key at all."""
    P, w, perm, nbr, wts, plan, s, copies, pts = inter_case()
    assert plan.rotation_amounts() == [] and plan.out_level == P.L - 2
    outs = layer.inter_ca_layer(P, plan, copies, pts)
    ref = wl.neighbor_reference(w, nbr, wts)
    for j, o in enumerate(outs):
        d = ckks.decode(P, ckks.decrypt(P, o, s), P.scale).real
        assert np.max(np.abs(d[perm] - ref[:, j])) < BOUND


def test_inter_ca_plan_on_plain_vectors():
    """The Inter-CA plan's masks and constants applied to plain slot vectors
    give sum_k w_k X[nbr_k] W to 1e-12 (the T3 check of this mode)."""
    P = ckks.Params(10, [60, 40, 40], [60], 1, 40)
    w = wl.make_workload(graph="er", V=30, deg=4.0, F=4, Fp=3, seed=2)
    perm = wl.random_order(w.V, P.slots, 2)
    nbr, wts = wl.sample_neighbors(w, 4, 2)
    plan = planner.build_inter_plan(P, P.L, nbr, wts, w.V, w.W, perm)
    ql = P.q[P.L]
    ref = wl.neighbor_reference(w, nbr, wts)
    for j in range(w.W.shape[1]):
        acc = np.zeros(P.slots)
        for k in range(nbr.shape[1]):
            Xk = np.where((nbr[:, k] >= 0)[:, None], w.X[np.maximum(nbr[:, k], 0)], 0.0)
            z = np.zeros(P.slots)
            for f in range(w.X.shape[1]):
                v = np.zeros(P.slots)
                v[perm] = Xk[:, f]
                z += plan.comb_consts[f][j] / ql * v
            acc += plan.masks[k].values * z
        assert np.max(np.abs(acc[perm] - ref[:, j])) < 1e-9


# ---------------------------------------------------------------- planted slips
def test_planted_slip_in_the_double_hoisted_form_fails(case, monkeypatch):
    """phi_g(c0) dropped from the double-hoisted outputs."""
    P, w, perm, plan, s, keys, cts, pts = case
    orig = ckks.keyswitch_ext

    def no_c0(params, ct, k, key, digits=None):
        u, c0g = orig(params, ct, k, key, digits)
        return u, np.zeros_like(c0g)
    monkeypatch.setattr(ckks, "keyswitch_ext", no_c0)
    z = layer.combination(P, plan, cts, keys, pts, 0)
    with pytest.raises(AssertionError):
        check_group_identity(P, plan, plan.groups[0], [z], keys, pts)


def test_planted_slip_in_the_plain_form_fails(case, monkeypatch):
    """The plain form's rotations taken the wrong way round."""
    P, w, perm, plan, s, keys, cts, pts = case
    orig = ckks.rotate
    amounts = plan.rotation_amounts()

    def wrong_way(params, ct, k, key, digits=None):
        k2 = (-k) % plan.M
        return orig(params, ct, k2, keys[k2] if k2 in amounts else key, digits)
    monkeypatch.setattr(ckks, "rotate", wrong_way)
    z = layer.combination(P, plan, cts, keys, pts, 0)
    with pytest.raises(AssertionError):
        check_group_identity(P, plan, plan.groups[0], [z], keys, pts)
    with pytest.raises(AssertionError):
        test_both_evaluators_decrypt_to_fp64(case, True)


def test_planted_slip_in_the_inter_ca_plan_fails(monkeypatch):
    """Neighbour weights attached to the wrong copies."""
    orig = planner.build_inter_plan

    def shifted(params, in_level, nbr, wts, V, W, perm):
        return orig(params, in_level, nbr, np.roll(np.asarray(wts), 1, axis=1), V, W, perm)
    monkeypatch.setattr(planner, "build_inter_plan", shifted)
    with pytest.raises(AssertionError):
        test_inter_ca_layer_decrypts_to_the_sampled_product()
