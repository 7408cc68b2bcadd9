"""Seeded synthetic inputs for the encrypted GCN layer.

This module holds no part of the method's arithmetic: it only draws graphs,
features, weights and node orders, and names the parameter sets.  Both the
library's tests/benchmark and the CPU oracle's tests take their inputs from
here, so the two sides always see identical inputs.

Graphs
  * "er":       Erdos-Renyi G(V, p = d/(V-1)), undirected.
  * "chung_lu": power-law expected degrees w_i ~ (i + i0)^(-1/(gamma-1)),
                scaled to mean degree d; V*d/2 edges drawn with both ends
                picked in proportion to w, then self-pairs and repeats
                removed (an edge-sampling form of the Chung-Lu model).
  A-hat = D^-1/2 (A + I) D^-1/2 (FP64), returned as CSR with sorted columns.

The public citation-benchmark datasets the paper evaluates on are not used:
these generators stand in for them with matching sizes, degree
distributions and feature densities.
"""
from dataclasses import dataclass

import numpy as np

# name -> CKKS parameters and workload shape (one GCN layer A-hat X W)
CONFIGS = {
    # toy, non-secure: 64-node ER graph, avg degree 4, X 64x16 U[-1,1],
    # W 16x8 N(0, 1/16); N = 2^12, scale 2^40, q = (60, 40, 40), one 60-bit
    # special prime, one prime per key-switching digit
    "toy": dict(log_n=12, q_bits=[60, 40, 40], p_bits=[60], alpha=1, log_scale=40,
                graph="er", V=64, deg=4.0, gamma=None, F=16, Fp=8,
                x="uniform", w="normal16", seed=0),
    # citation-graph-like: power law 2.5, 2708 nodes, avg degree 3.9,
    # X 2708x1433 binary ~1.3% ones, row-normalised; W 1433x16 Glorot;
    # N = 2^15, scale 2^40, 10 primes, dnum 3 (4 primes per digit, 4 special)
    "cora_like": dict(log_n=15, q_bits=[60] + [40] * 9, p_bits=[60] * 4, alpha=4,
                      log_scale=40, graph="chung_lu", V=2708, deg=3.9, gamma=2.5,
                      F=1433, Fp=16, x="binary", w="glorot", seed=0),
    # large: power law 2.5, 19717 nodes, avg degree 4.5, X 19717x500
    # TF-IDF-like (10% dense, Exp(1), row-normalised); W 500x16 Glorot;
    # N = 2^16, scale 2^45, 20 primes, dnum 5 (4 primes per digit, 4 special)
    "pubmed_like": dict(log_n=16, q_bits=[60] + [45] * 19, p_bits=[60] * 4, alpha=4,
                        log_scale=45, graph="chung_lu", V=19717, deg=4.5, gamma=2.5,
                        F=500, Fp=16, x="tfidf", w="glorot", seed=0),
}


# batched form: many single-layer queries of uneven size sharing one
# parameter set (N = 2^16, scale 2^45, 14 primes, dnum 4: 4 primes per
# digit, 4 special); each query's graph, features and weights come from
# batch_queries below
BATCH_PARAMS = dict(log_n=16, q_bits=[60] + [45] * 13, p_bits=[60] * 4, alpha=4, log_scale=45)


def batch_queries(n=32, first_seed=0):
    """n query workloads, seeds first_seed.. : power-law graphs of
    V ~ U{500..4000} nodes (mean degree 4) with exponent ~ U[2.1, 3.0],
    TF-IDF-like features F ~ U{64..512}, F' = 16, Glorot weights."""
    out = []
    for s in range(first_seed, first_seed + n):
        rng = np.random.default_rng(s)
        V = int(rng.integers(500, 4001))
        gamma = float(rng.uniform(2.1, 3.0))
        F = int(rng.integers(64, 513))
        out.append(make_workload(graph="chung_lu", V=V, deg=4.0, gamma=gamma, F=F, Fp=16,
                                 x="tfidf", w="glorot", seed=s))
    return out


def planner_graphs(seeds):
    """Workloads for training and judging the learned planner, one per seed:
    power-law graphs of V ~ U{1000..20000} nodes (mean degree 4) with
    exponent ~ U[2.1, 3.0], TF-IDF-like features F ~ U{128..1024}, F' = 16,
    Glorot weights (parameters: BATCH_PARAMS)."""
    out = []
    for s in seeds:
        rng = np.random.default_rng(s)
        V = int(rng.integers(1000, 20001))
        gamma = float(rng.uniform(2.1, 3.0))
        F = int(rng.integers(128, 1025))
        out.append(make_workload(graph="chung_lu", V=V, deg=4.0, gamma=gamma, F=F, Fp=16,
                                 x="tfidf", w="glorot", seed=s))
    return out


@dataclass
class Workload:
    V: int
    row_ptr: np.ndarray   # int32 [V+1]
    col: np.ndarray       # int32 [nnz]
    val: np.ndarray       # float64 [nnz]
    X: np.ndarray         # float64 [V][F]
    W: np.ndarray         # float64 [F][F']

    def dense_a(self):
        A = np.zeros((self.V, self.V))
        for v in range(self.V):
            for e in range(self.row_ptr[v], self.row_ptr[v + 1]):
                A[v, self.col[e]] += self.val[e]
        return A

    def reference_output(self):
        """FP64 A-hat X W."""
        XW = self.X @ self.W
        out = np.zeros((self.V, self.W.shape[1]))
        for v in range(self.V):
            s, e = self.row_ptr[v], self.row_ptr[v + 1]
            out[v] = self.val[s:e] @ XW[self.col[s:e]]
        return out

    def max_degree(self):
        return int(np.max(np.diff(self.row_ptr)))

    def mean_degree(self):
        return float(np.mean(np.diff(self.row_ptr)))


def er_edges(V, deg, rng):
    p = min(1.0, deg / max(1, V - 1))
    iu = np.triu_indices(V, 1)
    keep = rng.random(iu[0].size) < p
    return iu[0][keep], iu[1][keep]


def chung_lu_edges(V, deg, gamma, rng):
    i0 = 1.0
    w = (np.arange(V) + i0) ** (-1.0 / (gamma - 1.0))
    w *= deg * V / w.sum()
    m = int(round(V * deg / 2))
    prob = w / w.sum()
    a = rng.choice(V, size=m, p=prob)
    b = rng.choice(V, size=m, p=prob)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    keep = lo != hi
    pairs = np.unique(np.stack([lo[keep], hi[keep]], 1), axis=0)
    return pairs[:, 0], pairs[:, 1]


def normalized_adjacency(V, us, vs):
    """CSR of D^-1/2 (A + I) D^-1/2 for the undirected edge list (us, vs)."""
    rows = np.concatenate([us, vs, np.arange(V)])
    cols = np.concatenate([vs, us, np.arange(V)])
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    deg = np.bincount(rows, minlength=V).astype(np.float64)
    val = 1.0 / np.sqrt(deg[rows] * deg[cols])
    row_ptr = np.zeros(V + 1, dtype=np.int32)
    np.cumsum(np.bincount(rows, minlength=V), out=row_ptr[1:])
    return row_ptr, cols.astype(np.int32), val


def features(kind, V, F, rng):
    if kind == "uniform":
        return rng.uniform(-1.0, 1.0, size=(V, F))
    if kind == "binary":
        X = (rng.random((V, F)) < 0.013).astype(np.float64)
    elif kind == "tfidf":
        X = (rng.random((V, F)) < 0.10) * rng.exponential(1.0, size=(V, F))
    else:
        raise ValueError(kind)
    s = X.sum(axis=1, keepdims=True)
    return np.where(s > 0, X / np.where(s > 0, s, 1.0), 0.0)


def weights(kind, F, Fp, rng):
    if kind == "normal16":
        return rng.normal(0.0, 0.25, size=(F, Fp))
    if kind == "glorot":
        a = np.sqrt(6.0 / (F + Fp))
        return rng.uniform(-a, a, size=(F, Fp))
    raise ValueError(kind)


def make_workload(graph="er", V=64, deg=4.0, gamma=None, F=16, Fp=8, x="uniform",
                  w="normal16", seed=0, **_):
    rng = np.random.default_rng(seed)
    if graph == "er":
        us, vs = er_edges(V, deg, rng)
    elif graph == "chung_lu":
        us, vs = chung_lu_edges(V, deg, gamma, rng)
    else:
        raise ValueError(graph)
    row_ptr, col, val = normalized_adjacency(V, us, vs)
    X = features(x, V, F, rng)
    W = weights(w, F, Fp, rng)
    return Workload(V=V, row_ptr=row_ptr, col=col, val=val, X=X, W=W)


def config_workload(name, **over):
    cfg = dict(CONFIGS[name])
    cfg.update(over)
    return make_workload(**cfg)


# output classes of the second GCN layer (W2 is F' x C)
SECOND_LAYER_CLASSES = {"toy": 4, "cora_like": 7, "pubmed_like": 3}


def second_layer_weights(name, seed=None):
    """W2 (F' x C, Glorot-uniform) of a two-layer GCN on configuration name."""
    cfg = CONFIGS[name]
    rng = np.random.default_rng((cfg["seed"] if seed is None else seed) + 1)
    return weights("glorot", cfg["Fp"], SECOND_LAYER_CLASSES[name], rng)


def two_layer_reference(w, W2, first=None):
    """FP64 A-hat (H1)^2 W2 (square taken elementwise), H1 = A-hat X W1 unless
    the first layer's FP64 output is given (e.g. an Inter-CA layer's
    sum_k w_k X[nbr_k] W1)."""
    h = (w.reference_output() if first is None else first) ** 2
    XW = h @ W2
    out = np.zeros((w.V, W2.shape[1]))
    for v in range(w.V):
        s, e = w.row_ptr[v], w.row_ptr[v + 1]
        out[v] = w.val[s:e] @ XW[w.col[s:e]]
    return out


def sample_neighbors(w, n, seed):
    """GraphSage-style neighbourhoods for Inter-CA: node v itself, then up to
    n of its neighbours drawn without replacement; weights 1/(1 + drawn)
    (the MEAN aggregator).  Returns nbr [V][n+1] (-1 = none) and wts."""
    rng = np.random.default_rng(seed)
    nbr = np.full((w.V, n + 1), -1, dtype=np.int32)
    wts = np.zeros((w.V, n + 1))
    for v in range(w.V):
        nb = [int(u) for u in w.col[w.row_ptr[v]:w.row_ptr[v + 1]] if int(u) != v]
        pick = list(rng.choice(nb, size=min(n, len(nb)), replace=False)) if nb else []
        row = [v] + pick
        nbr[v, :len(row)] = row
        wts[v, :len(row)] = 1.0 / len(row)
    return nbr, wts


def full_neighbors(w):
    """Every neighbourhood of A-hat as Inter-CA copies: nbr [V][max row
    length] with the A-hat weights (the exact layer)."""
    n = w.max_degree()
    nbr = np.full((w.V, n), -1, dtype=np.int32)
    wts = np.zeros((w.V, n))
    for v in range(w.V):
        s, e = w.row_ptr[v], w.row_ptr[v + 1]
        nbr[v, :e - s] = w.col[s:e]
        wts[v, :e - s] = w.val[s:e]
    return nbr, wts


def neighbor_reference(w, nbr, wts):
    """FP64 sum_k wts[v][k] X[nbr[v][k]] W."""
    XW = w.X @ w.W
    out = np.zeros((w.V, w.W.shape[1]))
    for k in range(nbr.shape[1]):
        ok = nbr[:, k] >= 0
        out[ok] += wts[ok, k][:, None] * XW[nbr[ok, k]]
    return out


def random_order(V, size, seed):
    """A seeded injection of V nodes into [0, size)."""
    rng = np.random.default_rng(seed + 7919)
    return np.sort(rng.choice(size, size=V, replace=False))[rng.permutation(V)]


def identity_order(V):
    return np.arange(V, dtype=np.int64)


def random_words(primes, n, seed):
    """Uniform residues [len(primes)][n] (uint64), one row per prime: stand-in
    ciphertext limbs for word-for-word comparisons, where the values need no
    meaning.  numpy's PCG64 stream is the same on every platform."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, int(q), n, dtype=np.uint64) for q in primes])


def random_small_poly(n, bits, seed):
    """Integer coefficients uniform in [-2^bits, 2^bits] (int64): a stand-in
    plaintext given by its integers, so that both sides derive the same
    residues on any platform (no floating-point encoding in between)."""
    rng = np.random.default_rng(seed)
    return rng.integers(-(1 << bits), (1 << bits) + 1, n, dtype=np.int64)
