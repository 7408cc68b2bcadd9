"""The learned planner (the paper's packing and ordering choices, Sec. 3.2
and 3.4, made by a latency model instead of a search).

Every graph has candidate plans over the decisions the paper leaves to a
search: the packing t (the J(t) rule's choice, or its neighbour: t = 1
when the rule packs, else t = 2), the radix of the SpIntra-CA groups (2, 3
or 4 bits), and the node order (a seeded random order, or node order
optimisation, Alg. 1, with region size TH = 256 or 1024 and the regions
interleaved in search order or larger first).  The exhaustive planner builds
and runs every candidate and keeps the fastest.  The learned planner
computes each candidate's statistics on the host (fg_plan_features, no GPU
work), scores them with a three-layer perceptron trained on measured
latencies (fg_mlp_*, FP32 kernels on the GPU), and builds only the
candidate it predicts fastest.

  python -m paper_2506_10399_gb300.learn_planner measure OUT.jsonl [--budget S]
      layer latencies of every candidate of the held-out graphs (seeds
      2000-2019), then of the training graphs (seeds 1000-1199) until the
      time budget runs out; one JSON line per graph.  Plans are built for
      timing only (masks left zero: the kernels' work does not depend on the
      values), inputs are random residues.
  python -m paper_2506_10399_gb300.learn_planner train DATA.jsonl MODEL.json
      (the measured data of this repository: data/planner_latencies.jsonl)
      fit the model on the training graphs (GPU) and report, on the held-out
      graphs, the latency of its choices against the exhaustive planner's
      and against the default plan (radix 4, random order, t by the rule)
"""
import json
import sys
import time

import numpy as np

CANDIDATES = [
    dict(radix_bits=2, order="random", t="rule"),          # the default plan
    dict(radix_bits=3, order="random", t="rule"),
    dict(radix_bits=4, order="random", t="rule"),
    dict(radix_bits=2, order="random", t="alt"),
    dict(radix_bits=3, order="random", t="alt"),
    dict(radix_bits=2, order="noo", TH=256, region_order=0, t="rule"),
    dict(radix_bits=2, order="noo", TH=256, region_order=1, t="rule"),
    dict(radix_bits=2, order="noo", TH=1024, region_order=0, t="rule"),
    dict(radix_bits=3, order="noo", TH=256, region_order=1, t="rule"),
]
DEFAULT = 0            # radix 4 (2 bits), random order, t by the rule: the plain method's plan
HELD_OUT = list(range(2000, 2020))
TRAIN = list(range(1000, 1200))
HIDDEN = 64
DATA = __file__.rsplit("/", 1)[0] + "/data/planner_latencies.jsonl"
MODEL = __file__.rsplit("/", 1)[0] + "/data/planner_model.json"


def _fg():
    import __graft_entry__
    return __graft_entry__.build()


def packing_t(fg, P, w):
    """t of the J(t) rule (the planner's choice with t = 0)."""
    from . import workloads as wl
    f = fg.plan_features(P, w.row_ptr, w.col, w.val, w.W, wl.identity_order(w.V))
    return int(round(2.0 ** float(f[4])))


def candidate_t(cand, t_rule, V, M):
    """The candidate's t: the rule's, or its neighbour (1 when the rule
    packs, else 2 when two blocks of M/2 slots hold the graph); None when
    the neighbour does not exist."""
    if cand["t"] == "rule":
        return t_rule
    if t_rule > 1:
        return 1
    return 2 if 2 * V <= M else None


def candidate_perm(fg, wl, w, slots, cand, seed, cache=None):
    if cand["order"] == "noo":
        key = (slots, cand["TH"], cand["region_order"])
        if cache is not None and key in cache:
            return cache[key]
        perm, _ = fg.node_order(w.row_ptr, w.col, slots, cand["TH"], cand["region_order"])
        if cache is not None:
            cache[key] = perm
        return perm
    return wl.random_order(w.V, slots, seed)


def all_amounts(M):
    """Every rotation amount a plan of the candidates can need: signed digit
    amounts +-d 2^lo of the radix-2^r groups (r = 2, 3, 4) and the powers of
    two of the packing's rotate-and-sum."""
    am = set()
    logm = M.bit_length() - 1
    for r in sorted({c["radix_bits"] for c in CANDIDATES}):
        for lo in range(0, logm, r):
            for d in range(1, 1 << r):
                am.add((d << lo) % M)
                am.add((-(d << lo)) % M)
    am.update(1 << j for j in range(logm))
    am.discard(0)
    return am


def _record_amounts(rec, M):
    """Rotation amounts of a plan from its fg_plan_describe records."""
    V, F, Fp, t = int(rec[4]), int(rec[5]), int(rec[6]), int(rec[2])
    i = 13 + V
    am = set()
    if t == 1:
        i += F * Fp
    else:
        i += -(-F // t) * Fp
        nr = int(rec[i])
        am.update(int(k) % M for k in rec[i + 1:i + 1 + nr])
        i += 1 + nr
    for _ in range(int(rec[11])):
        nr = int(rec[i + 5])
        am.update(int(rec[i + 6 + 2 * r + 1]) % M for r in range(nr))
        i += 6 + 2 * nr
        i += 1 + 4 * int(rec[i])
    am.discard(0)
    return am


def measure(out_path, budget_s=1500.0):
    """Append to out_path the measurements of the graphs it does not hold
    yet (held-out seeds first), until the time budget runs out.  A candidate
    whose layer does not fit the device (out of memory, after the workspace
    was released once) is left out of its graph's record."""
    import os
    import torch
    fg = _fg()
    from . import workloads as wl
    P = wl.BATCH_PARAMS
    t0 = time.time()
    done = set()
    if os.path.exists(out_path):
        done = {json.loads(l)["seed"] for l in open(out_path) if l.strip()}
    ctx = fg.Context(**P)
    M = ctx.slots
    seeds = [s for s in HELD_OUT + TRAIN if s not in done]
    sk, evk = fg.keygen(ctx, 1, sorted(all_amounts(M)))
    keys = fg.load_evk(ctx, evk)
    del evk
    g = torch.Generator(device="cuda").manual_seed(0)

    def run_candidate(w, c, t, perm, xs):
        plan = fg.plan_build(ctx, w.row_ptr, w.col, w.val, w.W, perm, t=t,
                             radix_bits=c["radix_bits"], no_encode=True)
        try:
            feat = plan.features(w.row_ptr, w.col)
            info = plan.info()
            if t not in xs:
                # the timing does not depend on the values: random residues
                xs[t] = torch.randint(0, 1 << 40, (info["n_in"], 2, ctx.nq, ctx.n), dtype=torch.int64,
                                      device="cuda", generator=g)
            x = xs[t]
            out = torch.empty((info["n_out"], 2, info["out_level"] + 1, ctx.n), dtype=torch.int64,
                              device="cuda")
            fg.gcn_layer_axw(ctx, keys, plan, x, out=out)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            fg.gcn_layer_axw(ctx, keys, plan, x, out=out)
            e1.record()
            torch.cuda.synchronize()
            return {"t": t, "ms": e0.elapsed_time(e1), "features": [float(v) for v in feat],
                    "rotations": info["rotations"], "groups": info["n_groups"]}
        finally:
            plan.close()

    with open(out_path, "a") as f:
        for s in seeds:
            if time.time() - t0 > budget_s:
                break
            w = wl.planner_graphs([s])[0]
            t_rule = packing_t(fg, P, w)
            rows = []
            cache = {}
            xs = {}
            for ci, c in enumerate(CANDIDATES):
                t = candidate_t(c, t_rule, w.V, M)
                if t is None:
                    continue
                perm = candidate_perm(fg, wl, w, M // t, c, s, cache)
                for attempt in range(2):
                    try:
                        r = run_candidate(w, c, t, perm, xs)
                        r["cand"] = ci
                        rows.append(r)
                        break
                    except fg.FicgcnError as e:
                        if e.code not in (-4, -5) or "out of memory" not in str(e):
                            raise
                        xs.clear()
                        ctx.release_workspace()
                        torch.cuda.empty_cache()
            f.write(json.dumps({"seed": s, "V": w.V, "F": w.X.shape[1], "t_rule": t_rule, "cands": rows}) + "\n")
            f.flush()
            xs.clear()
            ctx.release_workspace()
            torch.cuda.empty_cache()
    print(json.dumps({"graphs_measured": sum(1 for _ in open(out_path)), "seconds": round(time.time() - t0)}))


def load(path):
    return [json.loads(l) for l in open(path)]


def complete(rows):
    """Graphs whose record holds the default candidate (needed to judge the
    gain over it)."""
    return [r for r in rows if any(c["cand"] == DEFAULT for c in r["cands"])]


def _xy(rows):
    """Features and targets: log2 latency relative to the mean over the
    graph's candidates (the choice only needs the order within a graph, and
    centring removes the graph-size scale the model would otherwise spend
    its capacity on)."""
    X = np.array([c["features"] for r in rows for c in r["cands"]], dtype=np.float64)
    y = []
    for r in rows:
        lg = np.log2(np.array([c["ms"] for c in r["cands"]], dtype=np.float64))
        y.extend(lg - lg.mean())
    return X, np.array(y)


def train(data_path, model_path, steps=3000, lr=3e-3, seed=0):
    fg = _fg()
    data = complete(load(data_path))
    held = [r for r in data if r["seed"] in HELD_OUT]
    tr = [r for r in data if r["seed"] not in HELD_OUT]
    X, y = _xy(tr)
    mu, sd = X.mean(axis=0), X.std(axis=0) + 1e-6
    rng = np.random.default_rng(seed)
    n_in = X.shape[1]
    shapes = [(n_in, HIDDEN), (HIDDEN,), (HIDDEN, HIDDEN), (HIDDEN,), (HIDDEN, 1), (1,)]
    init = np.concatenate([rng.normal(0, 1.0 / np.sqrt(s[0]), s).ravel() for s in shapes])
    m = fg.Mlp(n_in, HIDDEN, init.astype(np.float32))
    losses = m.train((X - mu) / sd, y, steps, lr)
    params = m.params()
    model = {"n_in": n_in, "hidden": HIDDEN, "mean": mu.tolist(), "std": sd.tolist(),
             "params": [float(v) for v in params], "train_graphs": len(tr), "train_rows": int(X.shape[0]),
             "final_loss": float(losses[-1]), "candidates": CANDIDATES}
    # the fallback margin: the default plan is kept unless a candidate is
    # predicted faster by more than the margin (log2 units), chosen on the
    # training graphs
    margins = [0.0, 0.02, 0.05, 0.1, 0.2, 0.3, 0.5]
    gains = [evaluate(m, mu, sd, tr, mg)["gain_vs_default"] for mg in margins]
    margin = margins[int(np.argmax(gains))]
    model["margin"] = margin
    model["train_gain_by_margin"] = dict(zip(map(str, margins), gains))
    report = evaluate(m, mu, sd, held, margin)
    model["held_out"] = report
    with open(model_path, "w") as f:
        json.dump(model, f)
    print(json.dumps({k: v for k, v in model.items() if k not in ("params", "mean", "std")}))
    return model


def load_model(path=MODEL):
    """(Mlp on the GPU, feature mean, feature scale) of a trained model."""
    fg = _fg()
    d = json.load(open(path))
    m = fg.Mlp(d["n_in"], d["hidden"], np.array(d["params"], dtype=np.float32))
    return m, np.array(d["mean"]), np.array(d["std"])


def default_ms(r):
    """Measured latency of a graph's default candidate."""
    return next(c["ms"] for c in r["cands"] if c["cand"] == DEFAULT)


def choose(m, mu, sd, features):
    """Index of the candidate the model predicts fastest (features as rows)."""
    b, _ = m.choose((np.asarray(features, dtype=np.float64) - mu) / sd)
    return b


def pick(pred, cands, margin):
    """The candidate the learned planner builds: the lowest prediction, unless
    it beats the default plan's prediction by no more than margin (log2
    latency), in which case the default (the exhaustive planner's fallback)."""
    b = int(np.argmin(pred))
    d = next(i for i, c in enumerate(cands) if c["cand"] == DEFAULT)
    return b if pred[b] < pred[d] - margin else d


def evaluate(m, mu, sd, rows, margin=0.0):
    """Per graph: measured latency of the learned planner's choice (pick),
    of the exhaustive planner's (the fastest candidate) and of the default
    plan."""
    chosen, best, default, hits = [], [], [], 0
    for r in rows:
        F = (np.array([c["features"] for c in r["cands"]]) - mu) / sd
        _, pred = m.choose(F)
        b = pick(pred, r["cands"], margin)
        ms = [c["ms"] for c in r["cands"]]
        chosen.append(ms[b])
        best.append(min(ms))
        default.append(default_ms(r))
        hits += int(ms[b] == min(ms))
    if not rows:
        return {}
    chosen, best, default = map(np.array, (chosen, best, default))
    return {"graphs": len(rows), "mean_ms_chosen": float(chosen.mean()),
            "mean_ms_exhaustive": float(best.mean()), "mean_ms_default": float(default.mean()),
            "gap_vs_exhaustive": float(chosen.sum() / best.sum() - 1.0),
            "gain_vs_default": float(1.0 - chosen.sum() / default.sum()),
            "picked_the_fastest": hits}


if __name__ == "__main__":
    cmd = sys.argv[1]
    if cmd == "measure":
        budget = float(sys.argv[sys.argv.index("--budget") + 1]) if "--budget" in sys.argv else 1500.0
        measure(sys.argv[2], budget)
    elif cmd == "train":
        train(sys.argv[2], sys.argv[3])
    else:
        raise SystemExit(__doc__)
