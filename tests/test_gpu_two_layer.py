"""The x^2 activation between GCN layers (CMult with relinearisation,
Sec. 2.1) and a two-layer encrypted GCN, bit for bit against the oracle."""
import numpy as np
import pytest

from oracle import ckks, layer, planner
from paper_2506_10399_gb300 import workloads as wl
from plan_records import oracle_records
from test_gpu_parity import PARAMS, parse_evk, rand_res, setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    return __graft_entry__.build()


@pytest.mark.parametrize("name", ["toy", "wide"])
def test_relin_key_matches_oracle(fg, name):
    ctx, P = setup(fg, name)
    seed = 21
    sk, evk = fg.keygen(ctx, seed, [1, 3], relin=True)
    ids, data = parse_evk(evk, P)
    assert ids[-1] == (fg.RELIN, 1) and [a for a, _ in ids[:-1]] == [1, 3]
    s = ckks.keygen_secret(P, seed)
    okey = ckks.keygen_relin(P, seed, s)
    keys = fg.load_evk(ctx, evk)
    for j, (b, a) in enumerate(okey):
        np.testing.assert_array_equal(data[-1, j, 0], b)
        np.testing.assert_array_equal(data[-1, j, 1], a)
        eb, ea = keys.export(fg.RELIN, j)
        np.testing.assert_array_equal(eb, b)


@pytest.mark.parametrize("name,level,same", [("toy", 2, True), ("toy", 1, False), ("multi", 6, True),
                                             ("multi", 3, False), ("wide", 7, True), ("deep", 12, False)])
def test_mul_relin_rescale_matches_oracle(fg, name, level, same):
    ctx, P = setup(fg, name)
    seed = 23
    sk, evk = fg.keygen(ctx, seed, [], relin=True)
    keys = fg.load_evk(ctx, evk)
    s = ckks.keygen_secret(P, seed)
    okey = ckks.keygen_relin(P, seed, s)
    rng = np.random.default_rng(level)
    a = np.stack([np.stack([rand_res(rng, P.q[:level + 1], P.n) for _ in range(2)]) for _ in range(2)])
    b = a if same else np.stack([np.stack([rand_res(rng, P.q[:level + 1], P.n) for _ in range(2)])
                                 for _ in range(2)])
    got = fg.mul_relin_rescale(ctx, keys, np.ascontiguousarray(a), np.ascontiguousarray(b), level)
    for c in range(2):
        np.testing.assert_array_equal(got[c], ckks.mul_relin_rescale(P, a[c], b[c], okey))


def test_mul_relin_rescale_needs_the_key(fg):
    ctx, P = setup(fg, "toy")
    _, evk = fg.keygen(ctx, 1, [1])
    keys = fg.load_evk(ctx, evk)
    a = np.zeros((2, 3, P.n), np.uint64)
    with pytest.raises(fg.FicgcnError) as e:
        fg.mul_relin_rescale(ctx, keys, a, a, 2)
    assert e.value.code == -3


def test_square_decrypts_to_square(fg):
    ctx, P = setup(fg, "wide")
    sk, evk = fg.keygen(ctx, 5, [], relin=True)
    keys = fg.load_evk(ctx, evk)
    rng = np.random.default_rng(0)
    z = rng.uniform(-1, 1, P.slots)
    lvl = 5
    ct = fg.encrypt(ctx, sk, 5, 0, fg.encode_plain(ctx, z, ctx.scale, lvl), lvl)
    sq = fg.mul_relin_rescale(ctx, keys, ct, ct, lvl)
    d = fg.decrypt_decode(ctx, sk, sq, lvl - 1, ctx.scale * ctx.scale / P.q[lvl])
    assert np.max(np.abs(d - z * z)) < 2 ** -20


def test_two_layer_gcn_bit_exact(fg):
    """Layer 1 (F -> F'), x^2, layer 2 (F' -> C) on one graph: every output
    residue equals the oracle's, and the decryption is within 2^-20 of
    A-hat (A-hat X W1)^2 W2."""
    ctx, P = setup(fg, "deep")
    w = wl.make_workload(graph="er", V=40, deg=3.0, F=5, Fp=3, seed=7)
    rng = np.random.default_rng(7)
    W2 = rng.normal(0, 0.5, (3, 2))
    perm = wl.random_order(w.V, P.slots, 7)
    op1 = planner.build_plan(P, P.L, w.row_ptr, w.col, w.val, w.V, w.W, perm, 1, 2, True, 6)
    plan1 = fg.plan_build(ctx, w.row_ptr, w.col, w.val, w.W, perm, t=1, radix_bits=2, min_out_level=6)
    np.testing.assert_array_equal(plan1.describe(), oracle_records(op1))
    l2 = op1.out_level - 1
    op2 = planner.build_plan(P, l2, w.row_ptr, w.col, w.val, w.V, W2, perm, 1, 2, True, 0)
    plan2 = fg.plan_build(ctx, w.row_ptr, w.col, w.val, W2, perm, t=1, radix_bits=2, in_level=l2)
    np.testing.assert_array_equal(plan2.describe(), oracle_records(op2))
    seed = 31
    amounts = sorted(set(plan1.rotation_amounts()) | set(plan2.rotation_amounts()))
    sk, evk = fg.keygen(ctx, seed, amounts, relin=True)
    keys = fg.load_evk(ctx, evk)
    s = ckks.keygen_secret(P, seed)
    okeys = {k: ckks.keygen_rotation(P, seed, s, k) for k in amounts}
    rkey = ckks.keygen_relin(P, seed, s)
    cts = []
    for f in range(w.X.shape[1]):
        v = np.zeros(P.slots)
        v[perm] = w.X[:, f]
        cts.append(ckks.encrypt(P, seed, f, ckks.encode(P, v, P.scale, P.L), s, P.L))
    pts1 = layer.encode_plan_masks(P, op1)
    pts2 = layer.encode_plan_masks(P, op2)
    for i, pt in enumerate(pts1):
        plan1.set_plaintext(i, pt)
    for i, pt in enumerate(pts2):
        plan2.set_plaintext(i, pt)
    h1, lvl1, sc1 = fg.gcn_layer_axw(ctx, keys, plan1, np.ascontiguousarray(np.stack(cts)))
    a1 = fg.mul_relin_rescale(ctx, keys, h1, h1, lvl1)
    out, lvl, _ = fg.gcn_layer_axw(ctx, keys, plan2, a1)
    # oracle, same steps
    o1 = layer.layer_axw(P, op1, cts, okeys, pts1)
    oa = [ckks.mul_relin_rescale(P, c, c, rkey) for c in o1]
    o2 = layer.layer_axw(P, op2, oa, okeys, pts2)
    for j in range(2):
        np.testing.assert_array_equal(out[j], o2[j])
    scale = sc1 * sc1 / P.q[lvl1]
    ref = w.reference_output()
    Xa = ref ** 2
    ref2 = np.zeros((w.V, 2))
    XW = Xa @ W2
    for v in range(w.V):
        s0, e0 = w.row_ptr[v], w.row_ptr[v + 1]
        ref2[v] = w.val[s0:e0] @ XW[w.col[s0:e0]]
    for j in range(2):
        d = fg.decrypt_decode(ctx, sk, np.ascontiguousarray(out[j]), lvl, scale)
        assert np.max(np.abs(d[perm] - ref2[:, j])) < 2 ** -20
