"""Batched layers: several queries of uneven size in flight at once (one
stream and workspace each), optionally captured into one CUDA graph, must
give the same ciphertexts word for word as running them one at a time; the
one-at-a-time path is itself bit-exact against the oracle (test_gpu_parity)."""
import numpy as np
import pytest

from paper_2506_10399_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

PARAMS = dict(log_n=13, q_bits=[60] + [45] * 7, p_bits=[60] * 3, alpha=3, log_scale=45)
QUERIES = [
    dict(graph="chung_lu", V=500, deg=4.0, gamma=2.1, F=64, Fp=4, x="tfidf", w="glorot", seed=0),
    dict(graph="chung_lu", V=1200, deg=3.5, gamma=2.7, F=24, Fp=4, x="binary", w="glorot", seed=1),
    dict(graph="er", V=300, deg=4.0, F=40, Fp=4, seed=2),
    dict(graph="chung_lu", V=2000, deg=4.5, gamma=3.0, F=16, Fp=4, x="tfidf", w="glorot", seed=3),
    dict(graph="chung_lu", V=800, deg=5.0, gamma=2.4, F=48, Fp=4, x="uniform", w="normal16", seed=4),
]


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    fg = __graft_entry__.build()
    ctx = fg.Context(**PARAMS)
    qs = []
    amounts = set()
    for i, wk in enumerate(QUERIES):
        w = wl.make_workload(**wk)
        t = fg.plan_build(ctx, w.row_ptr, w.col, w.val, w.W, wl.identity_order(w.V)).info()["t"]
        perm = wl.random_order(w.V, ctx.slots // t, 100 + i)
        plan = fg.plan_build(ctx, w.row_ptr, w.col, w.val, w.W, perm, t=t)
        amounts.update(plan.rotation_amounts())
        qs.append((w, perm, plan, t))
    sk, evk = fg.keygen(ctx, 9, sorted(amounts))   # one key set for every query
    keys = fg.load_evk(ctx, evk)
    data = []
    for i, (w, perm, plan, t) in enumerate(qs):
        info = plan.info()
        cin = torch.from_numpy(fg.pack_features(ctx, sk, 50 + i, w.X, perm, t).view(np.int64)).cuda()
        out = torch.empty((info["n_out"], 2, info["out_level"] + 1, ctx.n), dtype=torch.int64, device="cuda")
        data.append((cin, out))
    return fg, ctx, sk, keys, qs, data


def _one_at_a_time(fg, ctx, keys, qs, data):
    import torch
    res = []
    for (w, perm, plan, t), (cin, _) in zip(qs, data):
        out, lvl, _ = fg.gcn_layer_axw(ctx, keys, plan, cin)
        res.append((out.clone(), lvl))
    torch.cuda.synchronize()
    return res


@pytest.mark.parametrize("streams,graph", [(0, True), (2, False), (3, True)])
def test_batch_equals_one_at_a_time(env, streams, graph):
    fg, ctx, sk, keys, qs, data = env
    want = _one_at_a_time(fg, ctx, keys, qs, data)
    plans = [q[2] for q in qs]
    ins = [d[0] for d in data]
    outs = [d[1] for d in data]
    for rep in range(2):   # the second call replays the graph when one was captured
        for o in outs:
            o.zero_()
        lv, used = fg.gcn_layer_batch(ctx, keys, plans, ins, outs, streams=streams, graph=graph)
        assert 1 <= used <= max(streams, 8)
        if streams:
            assert used == min(streams, len(plans))
        for (o_w, l_w), o, l in zip(want, outs, lv):
            assert l == l_w
            assert bool((o == o_w).all())


def test_batch_decrypts_to_fp64(env):
    fg, ctx, sk, keys, qs, data = env
    plans = [q[2] for q in qs]
    lv, _ = fg.gcn_layer_batch(ctx, keys, plans, [d[0] for d in data], [d[1] for d in data])
    for (w, perm, plan, t), (cin, out), l in zip(qs, data, lv):
        ref = w.reference_output()
        for j in (0, w.W.shape[1] - 1):
            d = fg.decrypt_decode(ctx, sk, out[j].contiguous(), l, ctx.scale)
            assert np.max(np.abs(d[perm] - ref[:, j])) < 2 ** -20


def test_batch_rejects_host_buffers(env):
    fg, ctx, sk, keys, qs, data = env
    with pytest.raises(fg.FicgcnError) as e:
        fg.gcn_layer_batch(ctx, keys, [qs[0][2]], [data[0][0].cpu()], [data[0][1]])
    assert e.value.code == -1


def test_tuned_batch_equals_one_at_a_time(env):
    """The tuned form (launch configuration chosen by timing whole passes)
    gives the same words; the choice is one of the candidates and each
    candidate tried was timed."""
    fg, ctx, sk, keys, qs, data = env
    want = _one_at_a_time(fg, ctx, keys, qs, data)
    plans = [q[2] for q in qs]
    outs = [d[1] for d in data]
    for o in outs:
        o.zero_()
    fg.gcn_layer_batch(ctx, keys, plans, [d[0] for d in data], outs, streams=2, graph=True, tune=True)
    for (o_w, _), o in zip(want, outs):
        assert bool((o == o_w).all())
    cfg, ms = fg.batch_tuning(ctx)
    assert cfg["ks_split"] in (0, 1, 2) and cfg["ks_cols"] in (1, 2) and cfg["gmac_groups"] in (7, 4, 13)
    assert cfg["ntt_cols"] == 8 and cfg["ntt_rows"] == 8 and cfg["ntt_tw"] == 0   # N = 2^13: N = 2^16 forms stay
    assert cfg["kara"] in (0, 1)
    assert len(ms) == 8 and all(m > 0 for m in ms)   # default, 2 ks_split, ks_cols, 2 thresholds, kara, gmac_regs


def test_every_ntt16_tile_and_key_switch_bound_give_the_same_layer():
    """N = 2^16 (the tiles the tuner chooses among): the layer under each
    configuration the tuner can pick equals the default one word for word,
    through the batched entry point with tuning on."""
    import torch
    import __graft_entry__
    fg = __graft_entry__.build()
    P = dict(log_n=16, q_bits=[60] + [45] * 5, p_bits=[60] * 3, alpha=2, log_scale=45)
    ctx = fg.Context(**P)
    w = wl.make_workload(graph="chung_lu", V=3000, deg=4.0, gamma=2.5, F=12, Fp=2, x="tfidf", w="glorot",
                         seed=7)
    perm = wl.random_order(w.V, ctx.slots, 7)
    plan = fg.plan_build(ctx, w.row_ptr, w.col, w.val, w.W, perm, t=1, radix_bits=5)
    assert plan.info()["out_level"] == 1
    sk, evk = fg.keygen(ctx, 3, plan.rotation_amounts())
    keys = fg.load_evk(ctx, evk)
    cin = torch.from_numpy(fg.pack_features(ctx, sk, 4, w.X, perm, 1).view(np.int64)).cuda()
    want, lvl, _ = fg.gcn_layer_axw(ctx, keys, plan, cin)
    want = want.clone()
    for cfg in ((8, 16, 0, 0, 1, 0, 0, 7, 0), (16, 8, 0, 0, 1, 0, 0, 7, 0), (16, 16, 1, 0, 1, 0, 0, 7, 0),
                (8, 8, 1, 1, 2, 0, 0, 4, 1), (16, 16, 0, 1, 2, 0, 0, 13, 0), (16, 16, 0, 0, 1, 1, 0, 7, 0),
                (8, 8, 1, 0, 1, 1, 1, 7, 1), (16, 16, 0, 0, 1, 0, 1, 7, 0), (16, 16, 1, 0, 1, 1, 1, 7, 1), (16, 16, 0, 2, 1, 0, 0, 7, 0),
                (16, 16, 0, 0, 1, 0, 0, 7, 0, 0), (8, 8, 1, 1, 2, 1, 1, 4, 1, 0), (16, 16, 0, 2, 1, 0, 0, 13, 0, 0)):
        fg.set_tuning(ctx, *cfg)
        got, _, _ = fg.gcn_layer_axw(ctx, keys, plan, cin)
        assert bool((got == want).all()), cfg
    fg.set_tuning(ctx)
    out = torch.empty_like(want)
    fg.gcn_layer_batch(ctx, keys, [plan], [cin], [out], streams=1, graph=False, tune=True)
    assert bool((out == want).all())
    cfg, ms = fg.batch_tuning(ctx)
    assert len(ms) == 13 and cfg["ks_cols"] in (1, 2) and cfg["modup_fused"] in (0, 1) and cfg["ntt_cols"] in (16, 8) and cfg["ntt_rows"] in (16, 8) and cfg["ntt_tw"] in (0, 1)
    d = fg.decrypt_decode(ctx, sk, out[0].contiguous(), lvl, ctx.scale)
    assert np.max(np.abs(d[perm] - w.reference_output()[:, 0])) < 2 ** -20
    ctx.close()


@pytest.mark.parametrize("streams,graph", [(2, True), (3, False)])
def test_batch_from_page_locked_host_inputs(env, streams, graph):
    """Inputs in page-locked host memory (copied inside the batch, each
    stream with its own copy stream): the same words as one at a time."""
    import torch
    fg, ctx, sk, keys, qs, data = env
    want = _one_at_a_time(fg, ctx, keys, qs, data)
    plans = [q[2] for q in qs]
    ins = [d[0].cpu().pin_memory() for d in data]
    outs = [d[1] for d in data]
    for rep in range(2):
        for o in outs:
            o.zero_()
        fg.gcn_layer_batch(ctx, keys, plans, ins, outs, streams=streams, graph=graph)
        torch.cuda.synchronize()
        for (o_w, _), o in zip(want, outs):
            assert bool((o == o_w).all())


@pytest.mark.parametrize("where,streams,graph", [("host", 2, True), ("device", 3, False)])
def test_seeded_batch_equals_seeded_one_at_a_time(env, where, streams, graph):
    """Seeded client inputs (c0 parts; uniform halves regenerated on the
    device), page-locked host or device: the batch gives the same words as
    the queries one at a time through fg_gcn_layer_axw_seeded, on every
    call (the second replays the graph), and they decrypt to FP64."""
    import torch
    fg, ctx, sk, keys, qs, data = env
    plans = [q[2] for q in qs]
    seeds = [300 + i for i in range(len(qs))]
    ins = []
    for (w, perm, plan, t), sd in zip(qs, seeds):
        c0 = torch.from_numpy(fg.pack_features_seeded(ctx, sk, sd, w.X, perm, t).view(np.int64))
        ins.append(c0.pin_memory() if where == "host" else c0.cuda())
    want = []
    for plan, c0, sd in zip(plans, ins, seeds):
        out, lvl, _ = fg.gcn_layer_axw(ctx, keys, plan, c0.cuda(), seed=sd)
        want.append((out.clone(), lvl))
    outs = [torch.empty_like(o) for o, _ in want]
    for rep in range(2):
        for o in outs:
            o.zero_()
        lv, _ = fg.gcn_layer_batch(ctx, keys, plans, ins, outs, streams=streams, graph=graph, seeds=seeds)
        torch.cuda.synchronize()
        for (o_w, l_w), o, l in zip(want, outs, lv):
            assert l == l_w
            assert bool((o == o_w).all())
    for (w, perm, plan, t), o, l in zip(qs, outs, lv):
        d = fg.decrypt_decode(ctx, sk, o[0].contiguous(), l, ctx.scale)
        assert np.max(np.abs(d[perm] - w.reference_output()[:, 0])) < 2 ** -20
