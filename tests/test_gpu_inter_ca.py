"""Inter-CA (aggregation by PMult and Add over client-encrypted neighbour
copies): the plan equals the oracle planner's, every output residue equals
the oracle's, and the decryption is within 2^-20 of FP64."""
import numpy as np
import pytest

from oracle import ckks, layer, planner
from paper_2506_10399_gb300 import workloads as wl
from plan_records import oracle_records
from test_gpu_parity import setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    return __graft_entry__.build()


@pytest.mark.parametrize("name,mode", [("multi", "full"), ("deep", "sampled")])
def test_inter_ca_bit_exact(fg, name, mode):
    ctx, P = setup(fg, name)
    w = wl.make_workload(graph="chung_lu", V=60, deg=3.0, gamma=2.5, F=5, Fp=3, x="tfidf",
                         w="glorot", seed=12)
    nbr, wts = wl.full_neighbors(w) if mode == "full" else wl.sample_neighbors(w, 2, 3)
    perm = wl.random_order(w.V, P.slots, 12)
    op = planner.build_inter_plan(P, P.L, nbr, wts, w.V, w.W, perm)
    plan = fg.plan_build_inter(ctx, nbr, wts, w.W, perm)
    np.testing.assert_array_equal(plan.describe(), oracle_records(op))
    info = plan.info()
    assert info["n_in"] == nbr.shape[1] * w.X.shape[1] and info["out_level"] == P.L - 2
    seed = 77
    sk, evk = fg.keygen(ctx, seed, [])
    keys = fg.load_evk(ctx, evk)
    s = ckks.keygen_secret(P, seed)
    copies = []
    for k in range(nbr.shape[1]):
        Xk = np.where((nbr[:, k] >= 0)[:, None], w.X[np.maximum(nbr[:, k], 0)], 0.0)
        for f in range(w.X.shape[1]):
            v = np.zeros(P.slots)
            v[perm] = Xk[:, f]
            copies.append(ckks.encrypt(P, seed + k, f, ckks.encode(P, v, P.scale, P.L), s, P.L))
    pts = layer.encode_plan_masks(P, op)
    for i, pt in enumerate(pts):
        plan.set_plaintext(i, pt)
    out, lvl, scale = fg.gcn_layer_axw(ctx, keys, plan, np.ascontiguousarray(np.stack(copies)))
    want = layer.inter_ca_layer(P, op, copies, pts)
    for j in range(w.W.shape[1]):
        np.testing.assert_array_equal(out[j], want[j])
    ref = wl.neighbor_reference(w, nbr, wts)
    for j in range(w.W.shape[1]):
        d = fg.decrypt_decode(ctx, sk, np.ascontiguousarray(out[j]), lvl, scale)
        assert np.max(np.abs(d[perm] - ref[:, j])) < 2 ** -20
    if mode == "full":   # the exact layer: A-hat X W
        assert np.max(np.abs(ref - w.reference_output())) < 1e-12


def test_inter_ca_library_path(fg):
    """Client copies by the library's own packer (encoder, encryption)."""
    ctx, P = setup(fg, "wide")
    w = wl.make_workload(graph="chung_lu", V=900, deg=4.0, gamma=2.3, F=8, Fp=4, x="tfidf",
                         w="glorot", seed=4)
    nbr, wts = wl.sample_neighbors(w, 3, 5)
    perm = wl.random_order(w.V, P.slots, 4)
    plan = fg.plan_build_inter(ctx, nbr, wts, w.W, perm)
    sk, evk = fg.keygen(ctx, 8, [])
    keys = fg.load_evk(ctx, evk)
    cts = fg.pack_neighbor_copies(ctx, sk, 8, w.X, nbr, perm)
    out, lvl, scale = fg.gcn_layer_axw(ctx, keys, plan, cts)
    ref = wl.neighbor_reference(w, nbr, wts)
    for j in range(4):
        d = fg.decrypt_decode(ctx, sk, np.ascontiguousarray(out[j]), lvl, scale)
        assert np.max(np.abs(d[perm] - ref[:, j])) < 2 ** -20
