"""The learned planner's latency model on the GPU (FP32 kernels) against the
CPU reference (FP64): forward pass, gradients, Adam training, and the
choice among candidate plans."""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    return __graft_entry__.build()


def _case(seed, n=300, n_in=15, h=64):
    rng = np.random.default_rng(seed)
    params = [rng.normal(0, 1.0 / np.sqrt(s[0]), s).astype(np.float32).astype(np.float64)
              for s in mlp.sizes(n_in, h)]
    X = rng.normal(0, 1, (n, n_in)).astype(np.float32).astype(np.float64)
    y = rng.normal(0, 1, n).astype(np.float32).astype(np.float64)
    return params, X, y


@pytest.mark.parametrize("seed", [0, 1])
def test_forward_and_gradient_match_reference(fg, seed):
    params, X, y = _case(seed)
    m = fg.Mlp(15, 64, mlp.pack(params))
    f_ref, _ = mlp.forward(params, X)
    np.testing.assert_allclose(m.forward(X), f_ref, rtol=1e-4, atol=1e-4)
    loss, g = m.grad(X, y)
    l_ref, g_ref = mlp.loss_and_grads(params, X, y)
    assert abs(loss - l_ref) < 1e-4 * max(1.0, l_ref)
    g_ref = mlp.pack(g_ref)
    np.testing.assert_allclose(g, g_ref, rtol=2e-3, atol=2e-5 * np.max(np.abs(g_ref)))


def test_adam_training_follows_reference(fg):
    params, X, y = _case(2, n=200)
    m = fg.Mlp(15, 64, mlp.pack(params))
    losses = m.train(X, y, 30, 1e-3)
    p_ref, l_ref = mlp.adam(params, X, y, 30, 1e-3)
    np.testing.assert_allclose(losses, l_ref, rtol=1e-3)
    # Adam's step is about lr * sign(gradient): a gradient within FP32
    # rounding of zero may take the other sign, so a few parameters may
    # differ by up to 2 lr per step; all others agree closely
    close = np.isclose(m.params(), mlp.pack(p_ref), rtol=1e-3, atol=1e-5)
    assert close.mean() > 0.999
    assert losses[-1] < losses[0]


def test_choose_is_argmin_of_prediction(fg):
    params, X, _ = _case(3, n=9)
    m = fg.Mlp(15, 64, mlp.pack(params))
    best, pred = m.choose(X)
    f_ref, _ = mlp.forward(params, X)
    assert best == int(np.argmin(pred))
    np.testing.assert_allclose(pred, f_ref, rtol=1e-4, atol=1e-4)
    assert best == int(np.argmin(f_ref))


def test_trained_planner_choices_on_the_gpu(fg):
    """The trained model's choices by the GPU kernels equal the FP64
    reference's on every held-out graph."""
    import json
    import os
    from paper_2506_10399_gb300 import learn_planner as lp
    if not os.path.exists(lp.MODEL):
        pytest.skip("no trained model")
    d = json.load(open(lp.MODEL))
    m, mu, sd = lp.load_model()
    params = mlp.unpack(np.array(d["params"], dtype=np.float64), d["n_in"], d["hidden"])
    for r in lp.load(lp.DATA):
        if r["seed"] not in lp.HELD_OUT:
            continue
        F = np.array([c["features"] for c in r["cands"]])
        f, _ = mlp.forward(params, (F - mu) / sd)
        srt = np.sort(f)
        if srt[1] - srt[0] > 1e-4:        # a clear winner: both must pick it
            assert lp.choose(m, mu, sd, F) == int(np.argmin(f))


def test_features_of_a_built_plan_equal_the_host_features():
    """fg_plan_features_built (used while measuring) gives the statistics
    fg_plan_features computes from the same inputs."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    fg = __graft_entry__.build()
    from paper_2506_10399_gb300 import workloads as wl
    P = dict(log_n=13, q_bits=[60] + [45] * 7, p_bits=[60] * 2, alpha=4, log_scale=45)
    ctx = fg.Context(**P)
    w = wl.make_workload(graph="chung_lu", V=900, deg=4.0, gamma=2.5, F=20, Fp=4, seed=3)
    for t, r in ((1, 2), (2, 3)):
        perm = wl.random_order(w.V, ctx.slots // t, t)
        plan = fg.plan_build(ctx, w.row_ptr, w.col, w.val, w.W, perm, t=t, radix_bits=r, no_encode=True)
        want = fg.plan_features(P, w.row_ptr, w.col, w.val, w.W, perm, t=t, radix_bits=r)
        np.testing.assert_array_equal(plan.features(w.row_ptr, w.col), want)
