"""Seeded (compressed) client ciphertexts: only c0 crosses the host link and
the uniform part is regenerated on the device.  Checked word for word: the
regenerated part against the oracle's sampler, the client's c0 against the
oracle's seeded encryption of the same plaintext, and the layer on seeded
inputs (host and device, chunked t = 1 and packed t > 1) against the layer
on the expanded ciphertexts."""
import numpy as np
import pytest

from oracle import ckks
from paper_2506_10399_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

PARAMS = {
    "toy": dict(log_n=12, q_bits=[60, 40, 40], p_bits=[60], alpha=1, log_scale=40),
    "wide": dict(log_n=13, q_bits=[60] + [45] * 7, p_bits=[60] * 3, alpha=3, log_scale=45),
}


@pytest.fixture(scope="module")
def fg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    return __graft_entry__.build()


def params(fg, name):
    p = PARAMS[name]
    return fg.Context(**p), ckks.Params(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"])


@pytest.mark.parametrize("name,level", [("toy", 2), ("toy", 0), ("wide", 7), ("wide", 3)])
def test_regenerated_uniform_part_matches_oracle(fg, name, level):
    import torch
    ctx, P = params(fg, name)
    rng = np.random.default_rng(level)
    n, seed = 3, 41
    c0 = np.stack([np.stack([rng.integers(0, q, P.n, dtype=np.uint64) for q in P.q[:level + 1]])
                   for _ in range(n)])
    full = fg.expand_seeded(ctx, seed, c0)
    assert full.shape == (n, 2, level + 1, P.n)
    for b in range(n):
        np.testing.assert_array_equal(full[b, 0], c0[b])
        np.testing.assert_array_equal(full[b, 1], ckks.seeded_a(P, seed, b, level))
    dev = fg.expand_seeded(ctx, seed, torch.from_numpy(c0.view(np.int64)).cuda())
    np.testing.assert_array_equal(dev.cpu().numpy().view(np.uint64), full)
    ctx.close()


def test_seeded_packing_matches_oracle_encryption(fg):
    """c0 of every seeded ciphertext equals the oracle's encrypt_seeded of the
    same plaintext (the library's own encoding of the packed column, which
    fg_pack_features_seeded encrypts)."""
    ctx, P = params(fg, "wide")
    w = wl.make_workload(graph="er", V=150, deg=3.0, F=5, Fp=2, seed=4)
    t, seed = 2, 17
    perm = wl.random_order(w.V, P.slots // t, 5)
    sk, _ = fg.keygen(ctx, seed, [])
    s = ckks.keygen_secret(P, seed)
    c0 = fg.pack_features_seeded(ctx, sk, seed, w.X, perm, t)
    nb = -(-w.X.shape[1] // t)
    assert c0.shape == (nb, P.L + 1, P.n)
    B = P.slots // t
    for b in range(nb):
        z = np.zeros(P.slots)
        for k in range(t):
            f = b * t + k
            if f < w.X.shape[1]:
                z[k * B + perm] = w.X[:, f]
        pt = fg.encode_plain(ctx, z, P.scale, P.L)
        np.testing.assert_array_equal(c0[b], ckks.encrypt_seeded(P, seed, b, pt, s, P.L))
    full = fg.expand_seeded(ctx, seed, c0)
    d = fg.decrypt_decode(ctx, sk, np.ascontiguousarray(full[0]), P.L, P.scale)
    assert np.max(np.abs(d[perm] - w.X[:, 0])) < 2 ** -20
    ctx.close()


@pytest.mark.parametrize("F,t", [(130, 1), (24, 4)])
def test_layer_on_seeded_inputs_equals_the_expanded_layer(fg, F, t):
    """t = 1 with 130 columns: three 64-column chunks from host memory;
    t = 4: the packed inputs in one piece.  Host (numpy and page-locked)
    and device c0, all word for word the layer on the expanded inputs."""
    import torch
    ctx, P = params(fg, "wide")
    w = wl.make_workload(graph="chung_lu", V=600, deg=4.0, gamma=2.5, F=F, Fp=2, x="tfidf", w="glorot",
                         seed=8)
    perm = wl.random_order(w.V, P.slots // t, 9)
    plan = fg.plan_build(ctx, w.row_ptr, w.col, w.val, w.W, perm, t=t, radix_bits=3)
    sk, evk = fg.keygen(ctx, 3, plan.rotation_amounts())
    keys = fg.load_evk(ctx, evk)
    seed = 23
    c0 = fg.pack_features_seeded(ctx, sk, seed, w.X, perm, t)
    full = torch.from_numpy(fg.expand_seeded(ctx, seed, c0).view(np.int64)).cuda()
    want, lvl, scale = fg.gcn_layer_axw(ctx, keys, plan, full)
    want = want.cpu().numpy().view(np.uint64)
    for src in (c0, torch.from_numpy(c0.view(np.int64)).pin_memory(),
                torch.from_numpy(c0.view(np.int64)).cuda()):
        got, l2, _ = fg.gcn_layer_axw(ctx, keys, plan, src, seed=seed)
        got = got.cpu().numpy().view(np.uint64) if hasattr(got, "cpu") else got
        assert l2 == lvl
        np.testing.assert_array_equal(got, want)
    d = fg.decrypt_decode(ctx, sk, np.ascontiguousarray(want[0]), lvl, scale)
    assert np.max(np.abs(d[perm] - w.reference_output()[:, 0])) < 2 ** -20
    ctx.close()
