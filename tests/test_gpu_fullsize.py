"""The benchmark's own sizes (N = 2^16, 20 + 4 primes, dnum 5): sampled
operations bit for bit against the oracle (one rotation key, one rotation at
the top level, one rescale), and the whole benchmark layer through the
library checked by properties that hold at any size (decryption within
2^-20 of FP64 on sampled columns, output level and shape)."""
import numpy as np
import pytest

from oracle import ckks
from paper_2506_10399_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

CFG = wl.CONFIGS["pubmed_like"]


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    fg = __graft_entry__.build()
    ctx = fg.Context(**CFG)
    P = ckks.Params(CFG["log_n"], CFG["q_bits"], CFG["p_bits"], CFG["alpha"], CFG["log_scale"])
    return fg, ctx, P


def test_fullsize_rotation_key_and_rotation_match_oracle(env):
    fg, ctx, P = env
    seed, k = 31, 1234
    sk, evk = fg.keygen(ctx, seed, [k])
    keys = fg.load_evk(ctx, evk)
    s = ckks.keygen_secret(P, seed)
    okey = ckks.keygen_rotation(P, seed, s, k)
    eb, ea = keys.export(k, 2)
    np.testing.assert_array_equal(eb, okey[2][0])
    np.testing.assert_array_equal(ea, okey[2][1])
    rng = np.random.default_rng(5)
    z = rng.uniform(-1, 1, P.slots)
    lvl = P.L
    ct = ckks.encrypt(P, seed, 0, ckks.encode(P, z, P.scale, lvl), s, lvl)
    got = fg.rotate(ctx, keys, ct, lvl, k)
    np.testing.assert_array_equal(got, ckks.rotate(P, ct, k, okey))
    np.testing.assert_array_equal(fg.rescale(ctx, got, lvl), ckks.rescale_ct(P, got))


def test_fullsize_layer_decrypts_to_fp64(env):
    """The benchmark's layer (plan, keys, packing, launch configuration of
    bench.py) on its full inputs."""
    import torch
    fg, ctx, P = env
    w = wl.config_workload("pubmed_like")
    perm = wl.random_order(w.V, ctx.slots, 2025)
    plan = fg.plan_build(ctx, w.row_ptr, w.col, w.val, w.W, perm, t=1, radix_bits=2, min_out_level=10)
    info = plan.info()
    assert info["rotations"] == 4640 and info["out_level"] == 10
    sk, evk = fg.keygen(ctx, 2025, plan.rotation_amounts())
    keys = fg.load_evk(ctx, evk)
    x = torch.empty((info["n_in"], 2, ctx.nq, ctx.n), dtype=torch.int64, device="cuda")
    fg.pack_features(ctx, sk, 2025, w.X, perm, 1, out=x)
    out, lvl, scale = fg.gcn_layer_axw(ctx, keys, plan, x)
    assert tuple(out.shape) == (16, 2, 11, ctx.n) and lvl == 10
    ref = w.reference_output()
    for j in (0, 7, 15):
        d = fg.decrypt_decode(ctx, sk, out[j].contiguous(), lvl, scale)
        assert np.max(np.abs(d[perm] - ref[:, j])) < 2 ** -20


def test_cora_like_two_layer_decrypts_to_fp64():
    """The two-layer configuration at its full sizes (N = 2^15, 10 + 4 primes,
    dnum 3; V = 2708, F = 1433, F' = 16, 7 classes) on the exact A-hat: both
    layers SpIntra-CA at radix 32 (14-bit shifts in three groups), so the
    nine rescales are combination 1 + 3 groups, x^2 1 (CMult,
    relinearisation, rescale), combination 1 + 3 groups, and the output sits
    at level 0.  Every output column decrypts within 2^-20 of FP64
    A-hat (A-hat X W1)^2 W2."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    fg = __graft_entry__.build()
    cfg = wl.CONFIGS["cora_like"]
    ctx = fg.Context(**cfg)
    w = wl.config_workload("cora_like")
    W2 = wl.second_layer_weights("cora_like")
    perm = wl.random_order(w.V, ctx.slots, 5)
    plan1 = fg.plan_build(ctx, w.row_ptr, w.col, w.val, w.W, perm, t=1, radix_bits=5)
    i1 = plan1.info()
    assert i1["out_level"] == 5 and i1["n_groups"] == 3
    plan2 = fg.plan_build(ctx, w.row_ptr, w.col, w.val, W2, perm, t=1, radix_bits=5,
                          in_level=i1["out_level"] - 1)
    i2 = plan2.info()
    assert i2["out_level"] == 0 and i2["n_out"] == 7
    amounts = sorted(set(plan1.rotation_amounts()) | set(plan2.rotation_amounts()))
    sk, evk = fg.keygen(ctx, 5, amounts, relin=True)
    keys = fg.load_evk(ctx, evk)
    del evk
    x = torch.empty((i1["n_in"], 2, ctx.nq, ctx.n), dtype=torch.int64, device="cuda")
    fg.pack_features(ctx, sk, 5, w.X, perm, 1, out=x)
    h1 = torch.empty((i1["n_out"], 2, i1["out_level"] + 1, ctx.n), dtype=torch.int64, device="cuda")
    _, la, sc = fg.gcn_layer_axw(ctx, keys, plan1, x, out=h1)
    del x
    a1 = torch.empty((i1["n_out"], 2, la, ctx.n), dtype=torch.int64, device="cuda")
    fg.mul_relin_rescale(ctx, keys, h1, h1, la, out=a1)
    out = torch.empty((i2["n_out"], 2, i2["out_level"] + 1, ctx.n), dtype=torch.int64, device="cuda")
    _, lb, _ = fg.gcn_layer_axw(ctx, keys, plan2, a1, out=out)
    assert lb == 0
    scale = sc * sc / ctx.q[la]
    ref = wl.two_layer_reference(w, W2)
    for j in range(W2.shape[1]):
        d = fg.decrypt_decode(ctx, sk, out[j].contiguous(), lb, scale)
        assert np.max(np.abs(d[perm] - ref[:, j])) < 2 ** -20
