"""GPU path against the CPU oracle, element by element, through the C ABI.

Every ciphertext residue is compared bit for bit (all arithmetic is exact
mod q).  Where the GPU path and the oracle encode the same real values
independently (FP64 rounding of the canonical embedding) the inputs handed
to both are the oracle's encodings; the library's own encoder is checked
separately against the oracle's within one unit per coefficient.
"""
import math

import numpy as np
import pytest

from oracle import _ref, ckks, layer, planner
from paper_2506_10399_gb300 import workloads as wl
from plan_records import oracle_records

pytestmark = pytest.mark.gpu

PARAMS = {
    "toy": dict(log_n=12, q_bits=[60, 40, 40], p_bits=[60], alpha=1, log_scale=40),
    "multi": dict(log_n=11, q_bits=[60] + [40] * 6, p_bits=[60, 60], alpha=2, log_scale=40),
    "deep": dict(log_n=10, q_bits=[60] + [40] * 12, p_bits=[60], alpha=1, log_scale=40),
    "wide": dict(log_n=13, q_bits=[60] + [45] * 7, p_bits=[60] * 3, alpha=3, log_scale=45),
}


@pytest.fixture(scope="module")
def fg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    return __graft_entry__.build()


_cache = {}


def setup(fg, name):
    if name not in _cache:
        p = PARAMS[name]
        _cache[name] = (fg.Context(**p), ckks.Params(p["log_n"], p["q_bits"], p["p_bits"],
                                                     p["alpha"], p["log_scale"]))
    return _cache[name]


def rand_res(rng, primes, n):
    return np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in primes])


@pytest.mark.parametrize("name", list(PARAMS) + ["cora_like", "pubmed_like"])
def test_primes_match_oracle(fg, name):
    p = PARAMS.get(name) or wl.CONFIGS[name]
    ctx = fg.Context(**p)
    assert ctx.q == _ref.gen_primes(p["log_n"], p["q_bits"] + p["p_bits"])[:len(p["q_bits"])]
    assert ctx.p == _ref.gen_primes(p["log_n"], p["q_bits"] + p["p_bits"])[len(p["q_bits"]):]
    ctx.close()


@pytest.mark.parametrize("name,level", [("deep", 12), ("multi", 3), ("toy", 2), ("wide", 7)])
def test_poly_mul_matches_oracle(fg, name, level):
    ctx, P = setup(fg, name)
    rng = np.random.default_rng(level)
    a = rand_res(rng, P.q[:level + 1], P.n)
    b = rand_res(rng, P.q[:level + 1], P.n)
    got = fg.poly_mul(ctx, a, b, level)
    for i, q in enumerate(P.q[:level + 1]):
        np.testing.assert_array_equal(got[i], _ref.negacyclic_mul(a[i], b[i], q, P.psi(q)))


@pytest.mark.parametrize("log_n,pattern", [(15, "random"), (16, "random"), (16, "max")])
def test_poly_mul_large_n(fg, log_n, pattern):
    """N = 2^15 and 2^16 (the radix-16 path, lazy butterflies for the 45-bit
    primes); "max" sets every coefficient to q - 1, the largest inputs the
    lazy bounds must absorb."""
    p = dict(log_n=log_n, q_bits=[60, 45, 45], p_bits=[60], alpha=1, log_scale=45)
    ctx = fg.Context(**p)
    P = ckks.Params(log_n, p["q_bits"], p["p_bits"], 1, 45)
    rng = np.random.default_rng(log_n)
    if pattern == "max":
        a = np.stack([np.full(P.n, q - 1, dtype=np.uint64) for q in P.q])
        b = a.copy()
    else:
        a = rand_res(rng, P.q, P.n)
        b = rand_res(rng, P.q, P.n)
    got = fg.poly_mul(ctx, a, b, 2)
    for i in (0, 2):
        q = P.q[i]
        np.testing.assert_array_equal(got[i], _ref.negacyclic_mul(a[i], b[i], q, P.psi(q)))
    ctx.close()


@pytest.mark.parametrize("name", ["deep", "wide"])
def test_ntt_roundtrip_ragged_batches(fg, name):
    import torch
    ctx, P = setup(fg, name)
    for count, pidx in [(1, [0]), (7, [3, 1, 0, 2, 4, 1, 0]), (ctx.nq + ctx.np, list(range(ctx.nq + ctx.np)))]:
        primes = ctx.q + ctx.p
        rng = np.random.default_rng(count)
        host = np.stack([rng.integers(0, primes[pidx[c % len(pidx)]], P.n, dtype=np.uint64)
                         for c in range(count)])
        d = torch.from_numpy(host.view(np.int64).copy()).cuda()
        fg.ntt(ctx, d, pidx)
        fwd = d.cpu().numpy().view(np.uint64)
        assert not np.array_equal(fwd, host)
        assert all(fwd[c].max() < primes[pidx[c % len(pidx)]] for c in range(count))
        fg.ntt(ctx, d, pidx, inverse=True)
        np.testing.assert_array_equal(d.cpu().numpy().view(np.uint64), host)


def parse_evk(blob, P):
    import struct
    blob = bytes(blob) if not isinstance(blob, bytes) else blob
    assert blob[:8] == b"FGEVK001"
    ver, log_n, nq, np_, alpha, nk = struct.unpack_from("<6I", blob, 8)
    off = 8 + 24 + 8 * (nq + np_)
    ids = []
    for i in range(nk):
        ids.append(struct.unpack_from("<iI", blob, off))
        off += 8
    beta = -(-nq // alpha)
    kl = nq + np_
    data = np.frombuffer(blob, dtype=np.uint64, count=nk * beta * 2 * kl * P.n, offset=off)
    return ids, data.reshape(nk, beta, 2, kl, P.n)


@pytest.mark.parametrize("name", ["toy", "multi"])
def test_keygen_matches_oracle(fg, name):
    ctx, P = setup(fg, name)
    seed = 99
    amounts = [1, 5, P.slots - 3, P.slots // 2]
    sk, evk = fg.keygen(ctx, seed, amounts)
    s = ckks.keygen_secret(P, seed)
    np.testing.assert_array_equal(np.frombuffer(sk, np.int8, count=P.n, offset=16), s)
    ids, data = parse_evk(evk, P)
    assert [a for a, _ in ids] == sorted(amounts)
    keys = fg.load_evk(ctx, evk)
    for ki, (k, g) in enumerate(ids):
        assert g == P.galois(k)
        okey = ckks.keygen_rotation(P, seed, s, k)
        for j, (b, a) in enumerate(okey):
            np.testing.assert_array_equal(data[ki, j, 0], b)
            np.testing.assert_array_equal(data[ki, j, 1], a)
            eb, ea = keys.export(k, j)      # device copy survives NTT + Montgomery round trip
            np.testing.assert_array_equal(eb, b)
            np.testing.assert_array_equal(ea, a)


def test_corrupted_or_mismatched_evk_is_rejected(fg):
    ctx, P = setup(fg, "toy")
    _, evk = fg.keygen(ctx, 1, [1])
    bad = bytearray(evk)
    bad[100] ^= 1
    with pytest.raises(fg.FicgcnError) as e:
        fg.load_evk(ctx, bytes(bad))
    assert e.value.code == -3
    ctx2, _ = setup(fg, "multi")
    with pytest.raises(fg.FicgcnError) as e:
        fg.load_evk(ctx2, evk)
    assert e.value.code == -3


@pytest.mark.parametrize("name,level", [("toy", 2), ("multi", 6), ("multi", 0), ("wide", 4)])
def test_encrypt_decrypt_match_oracle(fg, name, level):
    ctx, P = setup(fg, name)
    seed = 7
    sk, _ = fg.keygen(ctx, seed, [])
    s = ckks.keygen_secret(P, seed)
    rng = np.random.default_rng(level)
    pt = ckks.encode(P, rng.uniform(-1, 1, P.slots), P.scale, level)
    ct = fg.encrypt(ctx, sk, seed, 3, pt, level)
    np.testing.assert_array_equal(ct, ckks.encrypt(P, seed, 3, pt, s, level))
    np.testing.assert_array_equal(fg.decrypt(ctx, sk, ct, level), ckks.decrypt(P, ct, s))


@pytest.mark.parametrize("name", ["toy", "wide"])
def test_encoder_within_one_unit_of_oracle(fg, name):
    ctx, P = setup(fg, name)
    rng = np.random.default_rng(3)
    for scale in (P.scale, float(P.q[1])):
        z = rng.uniform(-1, 1, P.slots)
        a = fg.encode_plain(ctx, z, scale, 1)
        b = ckks.encode(P, z, scale, 1)
        d = np.array([int(v) for v in ckks.crt_centered(P, ckks.sub_res(a, b, P.q[:2]))])
        assert np.max(np.abs(d)) <= 1 and np.mean(d != 0) < 0.01
        zz = ckks.decode(P, a, scale)
        assert np.max(np.abs(zz - z)) <= P.n / scale


@pytest.mark.parametrize("name,level", [("toy", 2), ("toy", 1), ("multi", 6), ("wide", 7)])
def test_rescale_matches_oracle(fg, name, level):
    ctx, P = setup(fg, name)
    rng = np.random.default_rng(level)
    ct = np.stack([rand_res(rng, P.q[:level + 1], P.n) for _ in range(2)])
    np.testing.assert_array_equal(fg.rescale(ctx, ct, level), ckks.rescale_ct(P, ct))


@pytest.mark.parametrize("name,level", [("toy", 2), ("toy", 0), ("multi", 6), ("multi", 3),
                                        ("wide", 7), ("wide", 2)])
def test_rotate_matches_oracle(fg, name, level):
    ctx, P = setup(fg, name)
    seed = 5
    ks = [1, -1, 3, 100, -257, P.slots // 2]
    sk, evk = fg.keygen(ctx, seed, ks)
    keys = fg.load_evk(ctx, evk)
    s = ckks.keygen_secret(P, seed)
    rng = np.random.default_rng(level)
    z = rng.uniform(-1, 1, P.slots)
    ct = ckks.encrypt(P, seed, 0, ckks.encode(P, z, P.scale, level), s, level)
    for k in ks:
        got = fg.rotate(ctx, keys, ct, level, k)
        want = ckks.rotate(P, ct, k, ckks.keygen_rotation(P, seed, s, k))
        np.testing.assert_array_equal(got, want)
    with pytest.raises(fg.FicgcnError) as e:
        fg.rotate(ctx, keys, ct, level, 2)
    assert e.value.code == -3


LAYERS = [
    # name, workload, t, radix, aoo, columns checked against the oracle
    ("deep", dict(graph="er", V=40, deg=3.0, F=5, Fp=3, seed=1), 1, 1, True, [0, 1, 2]),
    ("deep", dict(graph="er", V=40, deg=5.0, F=5, Fp=2, seed=2), 1, 2, False, [0, 1]),
    ("multi", dict(graph="chung_lu", V=150, deg=4.0, gamma=2.3, F=6, Fp=2, x="tfidf",
                   w="glorot", seed=3), 1, 3, True, [0, 1]),
    ("multi", dict(graph="er", V=30, deg=3.0, F=7, Fp=3, seed=4), 4, 3, True, [0, 2]),
    ("toy", dict(graph="er", V=64, deg=4.0, F=16, Fp=8, seed=0), 4, 11, True, [0, 7]),
    # groups of 8 and 11 outputs (three thread groups per group-MAC CTA) and of
    # 39 and 60 sources, 279 and 331 terms (each split over two launches)
    ("multi", dict(graph="er", V=1000, deg=4.0, F=4, Fp=2, seed=5), 1, 2, True, [0, 1]),
]


@pytest.mark.parametrize("li", range(len(LAYERS)))
def test_layer_bit_exact_vs_oracle(fg, li):
    name, wk, t, radix, aoo, cols = LAYERS[li]
    ctx, P = setup(fg, name)
    w = wl.make_workload(**wk)
    perm = wl.random_order(w.V, P.slots // t, li)
    op = planner.build_plan(P, P.L, w.row_ptr, w.col, w.val, w.V, w.W, perm, t, radix, aoo)
    plan = fg.plan_build(ctx, w.row_ptr, w.col, w.val, w.W, perm, t=t, radix_bits=radix, aoo=aoo)
    np.testing.assert_array_equal(plan.describe(), oracle_records(op))
    seed = 40 + li
    sk, evk = fg.keygen(ctx, seed, plan.rotation_amounts())
    keys = fg.load_evk(ctx, evk)
    s = ckks.keygen_secret(P, seed)
    okeys = {k: ckks.keygen_rotation(P, seed, s, k) for k in op.rotation_amounts()}
    nb = -(-w.X.shape[1] // t)
    B = P.slots // t
    cts = []
    for b in range(nb):
        v = np.zeros(P.slots)
        for kk in range(t):
            f = b * t + kk
            if f < w.X.shape[1]:
                v[kk * B + perm] = w.X[:, f]
        cts.append(ckks.encrypt(P, seed, b, ckks.encode(P, v, P.scale, P.L), s, P.L))
    pts = layer.encode_plan_masks(P, op)
    for i, pt in enumerate(pts):
        plan.set_plaintext(i, pt)
    out, lvl, scale = fg.gcn_layer_axw(ctx, keys, plan, np.ascontiguousarray(np.stack(cts)))
    assert lvl == op.out_level and out.shape == (w.W.shape[1], 2, lvl + 1, P.n)
    want = layer.layer_axw(P, op, cts, okeys, pts, columns=cols)
    for j, o in zip(cols, want):
        np.testing.assert_array_equal(out[j], o)
    ref = w.reference_output()
    for j in range(w.W.shape[1]):
        d = fg.decrypt_decode(ctx, sk, np.ascontiguousarray(out[j]), lvl, scale)
        assert np.max(np.abs(d[perm] - ref[:, j])) < 2 ** -20


@pytest.mark.parametrize("name,wk,t", [
    ("toy", dict(graph="er", V=64, deg=4.0, F=16, Fp=8, seed=0), 0),
    ("wide", dict(graph="chung_lu", V=1500, deg=4.5, gamma=2.5, F=12, Fp=4, x="tfidf", w="glorot",
                  seed=9), 1),
])
def test_layer_library_path_decrypts_to_fp64(fg, name, wk, t):
    """T2 through the library alone: its packing, encoder, planner and keys."""
    ctx, P = setup(fg, name)
    w = wl.make_workload(**wk)
    plan = fg.plan_build(ctx, w.row_ptr, w.col, w.val, w.W, wl.identity_order(w.V), t=t)
    info = plan.info()
    perm = wl.random_order(w.V, P.slots // info["t"], 11)
    plan = fg.plan_build(ctx, w.row_ptr, w.col, w.val, w.W, perm, t=info["t"])
    sk, evk = fg.keygen(ctx, 3, plan.rotation_amounts())
    keys = fg.load_evk(ctx, evk)
    cts = fg.pack_features(ctx, sk, 3, w.X, perm, info["t"])
    out, lvl, scale = fg.gcn_layer_axw(ctx, keys, plan, cts)
    ref = w.reference_output()
    for j in range(w.W.shape[1]):
        d = fg.decrypt_decode(ctx, sk, np.ascontiguousarray(out[j]), lvl, scale)
        assert np.max(np.abs(d[perm] - ref[:, j])) < 2 ** -20


def test_layer_argument_errors(fg):
    ctx, P = setup(fg, "deep")
    w = wl.make_workload(graph="er", V=20, deg=3.0, F=3, Fp=2, seed=1)
    perm = wl.random_order(w.V, P.slots, 1)
    plan = fg.plan_build(ctx, w.row_ptr, w.col, w.val, w.W, perm, t=1, radix_bits=2)
    ams = plan.rotation_amounts()
    sk, evk = fg.keygen(ctx, 1, ams[:-1])   # one key missing
    keys = fg.load_evk(ctx, evk)
    cts = fg.pack_features(ctx, sk, 1, w.X, perm, 1)
    with pytest.raises(fg.FicgcnError) as e:
        fg.gcn_layer_axw(ctx, keys, plan, cts)
    assert e.value.code == -3
    sk, evk = fg.keygen(ctx, 1, ams)
    keys = fg.load_evk(ctx, evk)
    with pytest.raises(fg.FicgcnError) as e:
        fg.gcn_layer_axw(ctx, keys, plan, np.ascontiguousarray(cts[:2]))
    assert e.value.code == -1


def test_layer_host_inputs_arrive_in_chunks(fg):
    """Host inputs of a t = 1 layer are copied in chunks of 64 columns, each
    chunk's combination starting when it arrives: the result equals the
    layer on the same inputs already in device memory."""
    import torch
    ctx, P = setup(fg, "multi")
    w = wl.make_workload(graph="er", V=50, deg=3.0, F=150, Fp=3, seed=21)
    perm = wl.random_order(w.V, P.slots, 21)
    plan = fg.plan_build(ctx, w.row_ptr, w.col, w.val, w.W, perm, t=1, radix_bits=2)
    sk, evk = fg.keygen(ctx, 21, plan.rotation_amounts())
    keys = fg.load_evk(ctx, evk)
    cts = fg.pack_features(ctx, sk, 21, w.X, perm, 1)
    host_out, lvl, scale = fg.gcn_layer_axw(ctx, keys, plan, cts)
    dev = torch.from_numpy(cts.view(np.int64)).cuda()
    dev_out, _, _ = fg.gcn_layer_axw(ctx, keys, plan, dev)
    np.testing.assert_array_equal(host_out, dev_out.cpu().numpy().view(np.uint64))
    ref = w.reference_output()
    d = fg.decrypt_decode(ctx, sk, np.ascontiguousarray(host_out[0]), lvl, scale)
    assert np.max(np.abs(d[perm] - ref[:, 0])) < 2 ** -20
