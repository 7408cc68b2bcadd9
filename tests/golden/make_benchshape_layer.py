"""Writes benchshape_layer.json: the oracle's output of one layer at the
benchmark's kernel shapes, for the word-for-word GPU test
(tests/test_gpu_benchshape.py).  Calls only oracle/ and the seeded input
generators.

The layer (paper Sec. 3.2-3.3, double-hoisted SpIntra-CA as the library
computes it): the pubmed_like parameters (N = 2^16, one 60-bit and nineteen
45-bit primes, four 60-bit special primes, 4 primes per key-switching digit,
so 5 digits and 23 extended limbs at level 18), F' = 16 output columns, t = 1,
radix-2 groups from level 18 with the output at level 10 or above.  The
graph is a 400-node Chung-Lu power law (exponent 2.5, mean degree 4.5) placed
at random in a window of 512 slots, which makes its groups open up to 11
lanes and read up to 47 sources (group MACs of three thread groups, sources
split over two launches); 136 input columns take the combination over two
128-column chunks.

Inputs are defined by integers so that both sides derive identical words on
any platform: every input ciphertext limb is a uniform residue, every mask
an integer polynomial with coefficients in [-2^44, 2^44] (reduced mod each
prime of its level and the special primes), keys come from the seeded
samplers.  The outputs are garbage as plaintexts; only their words matter.

Run from the repository root:  python tests/golden/make_benchshape_layer.py
(about ten minutes on eight cores).
"""
import concurrent.futures as cf
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ckks, layer, planner  # noqa: E402
from paper_2506_10399_gb300 import workloads as wl  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "benchshape_layer.json")

RECIPE = dict(
    config="pubmed_like",
    graph=dict(graph="chung_lu", V=400, deg=4.5, gamma=2.5, F=136, Fp=16, x="tfidf", w="glorot",
               seed=0),
    window=512, order_seed=2025, t=1, radix_bits=2, min_out_level=10,
    key_seed=2025, input_seed=100000, mask_seed=200000, mask_bits=44,
    columns=[0, 15], n_samples=64, sample_seed=99,
)


def params():
    c = wl.CONFIGS[RECIPE["config"]]
    return ckks.Params(c["log_n"], c["q_bits"], c["p_bits"], c["alpha"], c["log_scale"])


def case_inputs(P):
    """Workload, node order and the oracle's plan."""
    w = wl.make_workload(**RECIPE["graph"])
    perm = wl.random_order(w.V, RECIPE["window"], RECIPE["order_seed"])
    plan = planner.build_plan(P, P.L, w.row_ptr, w.col, w.val, w.V, w.W, perm, RECIPE["t"],
                              RECIPE["radix_bits"], min_out_level=RECIPE["min_out_level"])
    return w, perm, plan


def input_words(P, f):
    """Input ciphertext f: [2][L+1][N] uniform residues."""
    return np.stack([wl.random_words(P.q, P.n, RECIPE["input_seed"] + 2 * f + part)
                     for part in range(2)])


def mask_integers(P, i):
    return wl.random_small_poly(P.n, RECIPE["mask_bits"], RECIPE["mask_seed"] + i)


def oracle_mask(P, m, level):
    """The mask's residues over q_0..q_level and the special primes."""
    return np.stack([np.mod(m, np.int64(q)).astype(np.uint64) for q in P.ext_primes(level)])


def digest(ct):
    return hashlib.sha256(np.ascontiguousarray(ct, dtype="<u8").tobytes()).hexdigest()


def sample_positions(shape):
    rng = np.random.default_rng(RECIPE["sample_seed"])
    return [[int(rng.integers(0, shape[0])), int(rng.integers(0, shape[1])),
             int(rng.integers(0, shape[2]))] for _ in range(RECIPE["n_samples"])]


def plan_shape(plan):
    return [dict(level=g.level, n_in=g.n_in, n_out=g.n_out, rotations=len(g.rotations),
                 sources=len({(t.src, t.k) for t in g.terms}), terms=len(g.terms))
            for g in plan.groups]


def main():
    t0 = time.time()
    P = params()
    w, perm, plan = case_inputs(P)
    amounts = plan.rotation_amounts()
    s = ckks.keygen_secret(P, RECIPE["key_seed"])
    with cf.ThreadPoolExecutor(os.cpu_count()) as pool:
        keys = dict(zip(amounts, pool.map(
            lambda k: ckks.keygen_rotation(P, RECIPE["key_seed"], s, k), amounts)))
        print("keys: %d in %.0f s" % (len(keys), time.time() - t0), flush=True)
        cts = [input_words(P, f) for f in range(w.X.shape[1])]
        pts = [oracle_mask(P, mask_integers(P, i), m.level) for i, m in enumerate(plan.masks)]
        out = {}
        for j in RECIPE["columns"]:
            o = layer.layer_axw(P, plan, cts, keys, pts, columns=[j], pool=pool)[0]
            pos = sample_positions(o.shape)
            out[str(j)] = dict(sha256=digest(o), shape=list(o.shape),
                               samples=[p + [int(o[p[0], p[1], p[2]])] for p in pos])
            print("column %d in %.0f s" % (j, time.time() - t0), flush=True)
    doc = dict(
        what="oracle output of the benchmark-shaped layer (double-hoisted SpIntra-CA, "
             "paper Sec. 3.2-3.3); written by tests/golden/make_benchshape_layer.py",
        recipe=RECIPE, out_level=plan.out_level, n_masks=len(plan.masks),
        rotation_amounts=len(amounts), groups=plan_shape(plan), columns=out)
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote %s in %.0f s" % (OUT, time.time() - t0))


if __name__ == "__main__":
    main()
