"""GB300-native encrypted GCN layer A-hat X W under CKKS (FicGCN, ICML 2025).

Thin Python binding of the C ABI in include/ficgcn.h: every function here
only marshals arguments; all arithmetic runs in libficgcn.so (CUDA kernels
for sm_103a plus the host planner and encoder).  Buffers are numpy uint64
arrays (host) or torch int64 tensors holding the same 64-bit words (host or
CUDA); outputs follow the type of the main input unless `out` is given.

    ctx = Context(**params)
    sk, evk = keygen(ctx, seed, plan.rotation_amounts())
    keys = load_evk(ctx, evk)
    cts = pack_features(ctx, sk, seed, X, perm, t)
    out, level, scale = gcn_layer_axw(ctx, keys, plan, cts)
    Y = decrypt_decode(ctx, sk, out[j], level, scale)

Seeded synthetic inputs live in the submodule `workloads` (no arithmetic).
"""
import ctypes

import numpy as np

__all__ = ["Context", "Keys", "Plan", "FicgcnError", "ctx_create", "keygen", "load_evk",
           "encode_plain", "encrypt", "pack_features", "decrypt", "decrypt_decode",
           "plan_build", "plan_dry_run", "select_mode", "gcn_layer_axw", "rotate", "rescale", "poly_mul", "ntt"]


def _lib():
    from . import _native
    return _native


class FicgcnError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_lib().STATUS.get(code, "?"), code, msg))
        self.code = code


def _torch():
    import torch
    return torch


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """Raw pointer of a contiguous 64-bit numpy array or torch tensor."""
    if x is None:
        return None
    if _is_torch(x):
        assert x.is_contiguous() and x.element_size() == 8, "need a contiguous 64-bit tensor"
        return ctypes.c_void_p(x.data_ptr())
    assert isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"] and x.itemsize == 8, \
        "need a contiguous 64-bit numpy array"
    return ctypes.c_void_p(x.ctypes.data)


def _like(x, shape):
    if _is_torch(x):
        torch = _torch()
        return torch.empty(shape, dtype=torch.int64, device=x.device)
    return np.empty(shape, dtype=np.uint64)


def _check(ctx, rc):
    if rc != 0:
        msg = _lib().lib.fg_last_error(ctx._h if ctx is not None else None)
        raise FicgcnError(rc, (msg or b"").decode())


class Context:
    """fg_ctx: parameters, primes and device tables on the current CUDA device."""

    def __init__(self, log_n, q_bits, p_bits, alpha, log_scale, stream=None, **_):
        nat = _lib()
        self.log_n, self.n, self.slots = log_n, 1 << log_n, 1 << (log_n - 1)
        self.nq, self.np = len(q_bits), len(p_bits)
        self.alpha, self.log_scale, self.scale = alpha, log_scale, float(2.0 ** log_scale)
        qb = (ctypes.c_int * len(q_bits))(*q_bits)
        pb = (ctypes.c_int * len(p_bits))(*p_bits)
        prm = nat.Params(log_n, len(q_bits), qb, len(p_bits), pb, alpha, float(log_scale))
        if stream is None:
            try:
                torch = _torch()
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                stream = None
        self._stream = stream
        h = ctypes.c_void_p()
        self._h = None
        rc = nat.lib.fg_ctx_create(ctypes.byref(prm), ctypes.c_void_p(stream or 0), ctypes.byref(h))
        if rc != 0:
            raise FicgcnError(rc, "context creation failed: " + nat.lib.fg_last_error(None).decode())
        self._h = h
        q = np.zeros(self.nq, np.uint64)
        p = np.zeros(self.np, np.uint64)
        nat.lib.fg_ctx_primes(h, _ptr(q), _ptr(p))
        self.q, self.p = [int(v) for v in q], [int(v) for v in p]
        self.L = self.nq - 1

    def device_bytes(self):
        b = ctypes.c_size_t()
        _check(self, _lib().lib.fg_ctx_device_bytes(self._h, ctypes.byref(b)))
        return b.value

    def release_workspace(self):
        """Free the scratch buffers the context keeps between calls."""
        _check(self, _lib().lib.fg_ctx_release_workspace(self._h))

    def time_kernels(self, kernel_class):
        """Start CUDA-event timing of one kernel class (None stops)."""
        _check(self, _lib().lib.fg_ctx_time_kernels(
            self._h, kernel_class.encode() if kernel_class else None))

    def kernel_times(self):
        """(device ms, calls, algorithmic bytes) of the timed class since the last read."""
        ms, n, by = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        _check(self, _lib().lib.fg_ctx_kernel_times(self._h, ctypes.byref(ms), ctypes.byref(n),
                                                    ctypes.byref(by)))
        return ms.value, n.value, by.value

    def launch_count(self):
        n = ctypes.c_int64()
        _check(self, _lib().lib.fg_ctx_launch_count(self._h, ctypes.byref(n)))
        return n.value

    def close(self):
        if self._h is not None:
            _lib().lib.fg_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ctx_create(**params):
    return Context(**params)


class Keys:
    """fg_keys: rotation keys on the device."""

    def __init__(self, ctx, h):
        self.ctx, self._h = ctx, h

    def export(self, amount, digit):
        """Coefficient-domain (b, a) of one digit of one key, [L+1+K][N] each."""
        kl = self.ctx.nq + self.ctx.np
        b = np.zeros((kl, self.ctx.n), np.uint64)
        a = np.zeros((kl, self.ctx.n), np.uint64)
        _check(self.ctx, _lib().lib.fg_keys_export(self._h, int(amount), int(digit), _ptr(b), _ptr(a)))
        return b, a

    def close(self):
        if self._h is not None:
            _lib().lib.fg_keys_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


RELIN = -1   # evk entry of the relinearisation key


def keygen(ctx, seed, rot_amounts, relin=False):
    """(secret-key blob as bytes, evaluation-key blob as a numpy uint8 array);
    relin=True adds the relinearisation key for mul_relin_rescale."""
    nat = _lib()
    am = np.ascontiguousarray(np.array(list(rot_amounts), dtype=np.int32))
    skb, skl, evb, evl = ctypes.c_void_p(), ctypes.c_size_t(), ctypes.c_void_p(), ctypes.c_size_t()
    _check(ctx, nat.lib.fg_keygen(ctx._h, int(seed), am.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                  len(am), 1 if relin else 0, ctypes.byref(skb), ctypes.byref(skl),
                                  ctypes.byref(evb), ctypes.byref(evl)))
    sk = _copy_blob(skb, skl.value).tobytes()
    evk = _copy_blob(evb, evl.value)
    nat.lib.fg_free(skb)
    nat.lib.fg_free(evb)
    return sk, evk


def _copy_blob(ptr, n):
    """Copy a library-owned blob (any size; ctypes.string_at takes a C int)."""
    if n == 0:
        return np.zeros(0, np.uint8)
    return np.frombuffer((ctypes.c_uint8 * n).from_address(ptr.value), dtype=np.uint8).copy()


def _blob_arg(b):
    if isinstance(b, np.ndarray):
        assert b.dtype == np.uint8 and b.flags["C_CONTIGUOUS"]
        return ctypes.c_void_p(b.ctypes.data), b.size
    return b, len(b)


def load_evk(ctx, evk):
    """Keys from an evk blob (bytes or a numpy uint8 array, as keygen returns)."""
    h = ctypes.c_void_p()
    ptr, n = _blob_arg(evk)
    _check(ctx, _lib().lib.fg_load_evk(ctx._h, ptr, n, ctypes.byref(h)))
    return Keys(ctx, h)


def encode_plain(ctx, slots, scale, level, out=None):
    z = np.ascontiguousarray(np.asarray(slots, dtype=np.float64))
    if out is None:
        out = np.empty((level + 1, ctx.n), np.uint64)
    _check(ctx, _lib().lib.fg_encode_plain(ctx._h, _ptr(z), z.size, float(scale), level, _ptr(out)))
    return out


def encrypt(ctx, sk, seed, index, pt, level, out=None):
    if out is None:
        out = _like(pt, (2, level + 1, ctx.n))
    _check(ctx, _lib().lib.fg_encrypt(ctx._h, sk, len(sk), int(seed), int(index), _ptr(pt), level,
                                      _ptr(out)))
    return out


def pack_features(ctx, sk, seed, X, perm, t, out=None):
    """ceil(F/t) ciphertexts [2][L+1][N] of the column-packed features."""
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    perm = np.ascontiguousarray(np.asarray(perm, dtype=np.int32))
    V, F = X.shape
    nb = -(-F // t)
    if out is None:
        out = np.empty((nb, 2, ctx.nq, ctx.n), np.uint64)
    n = ctypes.c_int()
    _check(ctx, _lib().lib.fg_pack_features(ctx._h, sk, len(sk), int(seed), _ptr(X), V, F,
                                            ctypes.c_void_p(perm.ctypes.data), t, _ptr(out),
                                            ctypes.byref(n)))
    return out


def pack_features_seeded(ctx, sk, seed, X, perm, t, out=None):
    """Seeded form of pack_features: the c0 parts [ceil(F/t)][L+1][N] only;
    ciphertext b's uniform part is regenerated from (seed, b) by
    expand_seeded or by gcn_layer_axw(..., seed=seed)."""
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    perm = np.ascontiguousarray(np.asarray(perm, dtype=np.int32))
    V, F = X.shape
    nb = -(-F // t)
    if out is None:
        out = np.empty((nb, ctx.nq, ctx.n), np.uint64)
    n = ctypes.c_int()
    _check(ctx, _lib().lib.fg_pack_features_seeded(ctx._h, sk, len(sk), int(seed), _ptr(X), V, F,
                                                   ctypes.c_void_p(perm.ctypes.data), t, _ptr(out),
                                                   ctypes.byref(n)))
    return out


def expand_seeded(ctx, seed, c0, out=None):
    """Full ciphertexts [n][2][l+1][N] of seeded ones (c0: [n][l+1][N])."""
    n, nl = int(c0.shape[0]), int(c0.shape[1])
    if out is None:
        out = _like(c0, (n, 2, nl, ctx.n))
    _check(ctx, _lib().lib.fg_expand_seeded(ctx._h, int(seed), _ptr(c0), n, nl - 1, _ptr(out)))
    return out


def decrypt(ctx, sk, ct, level, out=None):
    if out is None:
        out = _like(ct, (level + 1, ctx.n))
    _check(ctx, _lib().lib.fg_decrypt(ctx._h, sk, len(sk), _ptr(ct), level, _ptr(out)))
    return out


def decrypt_decode(ctx, sk, ct, level, scale):
    out = np.empty(ctx.slots, np.float64)
    _check(ctx, _lib().lib.fg_decrypt_decode(ctx._h, sk, len(sk), _ptr(ct), level, float(scale),
                                             _ptr(out)))
    return out


class Plan:
    """fg_plan: the layer's packing, SpIntra-CA schedule and device masks."""

    def __init__(self, ctx, h):
        self.ctx, self._h = ctx, h

    def info(self):
        i = _lib().PlanInfo()
        _check(self.ctx, _lib().lib.fg_plan_info(self._h, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in i._fields_}

    def rotation_amounts(self):
        n = ctypes.c_int()
        _lib().lib.fg_plan_rotation_amounts(self._h, None, 0, ctypes.byref(n))
        out = np.zeros(max(1, n.value), np.int32)
        _check(self.ctx, _lib().lib.fg_plan_rotation_amounts(self._h, ctypes.c_void_p(out.ctypes.data),
                                                             n.value, ctypes.byref(n)))
        return [int(v) for v in out[:n.value]]

    def describe(self):
        ln = ctypes.c_size_t()
        _check(self.ctx, _lib().lib.fg_plan_describe(self._h, None, 0, ctypes.byref(ln)))
        out = np.zeros(ln.value, np.int64)
        _check(self.ctx, _lib().lib.fg_plan_describe(self._h, _ptr(out), ln.value, ctypes.byref(ln)))
        return out

    def features(self, row_ptr, col):
        """The learned planner's statistics of this plan (its graph's CSR)."""
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        col = np.ascontiguousarray(col, dtype=np.int32)
        out = np.zeros(N_PLAN_FEATURES, np.float32)
        _check(self.ctx, _lib().lib.fg_plan_features_built(self._h, ctypes.c_void_p(row_ptr.ctypes.data),
                                                           ctypes.c_void_p(col.ctypes.data),
                                                           ctypes.c_void_p(out.ctypes.data)))
        return out

    def set_plaintext(self, mask, coeffs):
        coeffs = coeffs if _is_torch(coeffs) else np.ascontiguousarray(coeffs, dtype=np.uint64)
        _check(self.ctx, _lib().lib.fg_plan_set_plaintext(self._h, int(mask), _ptr(coeffs)))

    def close(self):
        if self._h is not None:
            _lib().lib.fg_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_build_inter(ctx, nbr, wts, W, perm, min_out_level=0, in_level=0):
    """Inter-CA plan: nbr, wts [V][n] (neighbour index or -1, its weight)."""
    nat = _lib()
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    wts = np.ascontiguousarray(wts, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    V, n = nbr.shape
    F, Fp = W.shape
    o = nat.PlanOpts(1, 0, 1, int(min_out_level), 0, int(in_level), 0)
    h = ctypes.c_void_p()
    _check(ctx, nat.lib.fg_plan_build_inter(ctx._h, ctypes.c_void_p(nbr.ctypes.data), _ptr(wts), V, n,
                                            _ptr(W), F, Fp, ctypes.c_void_p(perm.ctypes.data),
                                            ctypes.byref(o), ctypes.byref(h)))
    return Plan(ctx, h)


def pack_neighbor_copies(ctx, sk, seed, X, nbr, perm, out=None):
    """The client's Inter-CA input (fg_pack_neighbor_copies): for every
    neighbour slot k, the rows nbr[:, k] of X (zero where nbr is -1) packed
    as pack_features does, copy k encrypted under seed + k;
    [n*F][2][L+1][N], copy-major."""
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    nbr = np.ascontiguousarray(np.asarray(nbr), dtype=np.int32)
    perm = np.ascontiguousarray(np.asarray(perm, dtype=np.int32))
    V, F = X.shape
    n = nbr.shape[1]
    if out is None:
        out = np.empty((n * F, 2, ctx.nq, ctx.n), np.uint64)
    _check(ctx, _lib().lib.fg_pack_neighbor_copies(ctx._h, sk, len(sk), int(seed), _ptr(X), V, F,
                                                   ctypes.c_void_p(nbr.ctypes.data), n,
                                                   ctypes.c_void_p(perm.ctypes.data), _ptr(out)))
    return out


def plan_build(ctx, row_ptr, col, val, W, perm, t=0, radix_bits=0, aoo=True, min_out_level=0,
               n_sampled=0, in_level=0, no_encode=False):
    """Plan of one layer; no_encode leaves every mask zero (a plan for timing
    only)."""
    nat = _lib()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    V = row_ptr.size - 1
    F, Fp = W.shape
    o = nat.PlanOpts(int(t), int(radix_bits), 1 if aoo else 0, int(min_out_level), int(n_sampled),
                     int(in_level), 1 if no_encode else 0)
    h = ctypes.c_void_p()
    _check(ctx, nat.lib.fg_plan_build(ctx._h, ctypes.c_void_p(row_ptr.ctypes.data),
                                      ctypes.c_void_p(col.ctypes.data), _ptr(val), V, _ptr(W), F, Fp,
                                      ctypes.c_void_p(perm.ctypes.data), ctypes.byref(o),
                                      ctypes.byref(h)))
    return Plan(ctx, h)


def node_order(row_ptr, col, slots, th, region_order=0):
    """(perm node -> slot, number of regions) by node order optimisation;
    region_order 1 interleaves larger regions first."""
    nat = _lib()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    V = row_ptr.size - 1
    perm = np.empty(V, np.int32)
    nr = ctypes.c_int()
    rc = nat.lib.fg_node_order_ex(ctypes.c_void_p(row_ptr.ctypes.data), ctypes.c_void_p(col.ctypes.data),
                                  V, int(slots), int(th), int(region_order),
                                  ctypes.c_void_p(perm.ctypes.data), ctypes.byref(nr))
    if rc != 0:
        raise FicgcnError(rc, "node order failed")
    return perm, nr.value


def plan_dry_run(params, row_ptr, col, val, W, perm, t=0, radix_bits=0, aoo=True,
                 min_out_level=0, n_sampled=0, in_level=0):
    """Plan records (as Plan.describe()) computed on the host only, no device."""
    nat = _lib()
    q_bits, p_bits = params["q_bits"], params["p_bits"]
    qb = (ctypes.c_int * len(q_bits))(*q_bits)
    pb = (ctypes.c_int * len(p_bits))(*p_bits)
    prm = nat.Params(params["log_n"], len(q_bits), qb, len(p_bits), pb, params["alpha"],
                     float(params["log_scale"]))
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    F, Fp = W.shape
    o = nat.PlanOpts(int(t), int(radix_bits), 1 if aoo else 0, int(min_out_level), int(n_sampled),
                     int(in_level), 0)
    args = [ctypes.byref(prm), ctypes.c_void_p(row_ptr.ctypes.data), ctypes.c_void_p(col.ctypes.data),
            _ptr(val), row_ptr.size - 1, _ptr(W), F, Fp, ctypes.c_void_p(perm.ctypes.data),
            ctypes.byref(o)]
    ln = ctypes.c_size_t()
    rc = nat.lib.fg_plan_dry_run(*args, None, 0, ctypes.byref(ln))
    if rc != 0:
        raise FicgcnError(rc, "planning failed")
    out = np.zeros(ln.value, np.int64)
    rc = nat.lib.fg_plan_dry_run(*args, _ptr(out), ln.value, ctypes.byref(ln))
    if rc != 0:
        raise FicgcnError(rc, "planning failed")
    return out


def gcn_layer_axw(ctx, keys, plan, in_cts, out=None, seed=None):
    """(output ciphertexts [F'][2][l+1][N], output level l, scale).  With
    seed given, in_cts are the c0 parts [n][in_level+1][N] of seeded
    ciphertexts (pack_features_seeded)."""
    info = plan.info()
    if out is None:
        out = _like(in_cts, (info["n_out"], 2, info["out_level"] + 1, ctx.n))
    assert int(in_cts.shape[-1]) == ctx.n and int(in_cts.shape[-2]) == info["in_level"] + 1, \
        "inputs must be [n][2][in_level+1][N] ([n][in_level+1][N] when seeded)"
    assert (seed is None) == (in_cts.ndim == 4), "seeded inputs are c0 parts [n][in_level+1][N]"
    lvl, sc = ctypes.c_int(), ctypes.c_double()
    if seed is None:
        _check(ctx, _lib().lib.fg_gcn_layer_axw(ctx._h, keys._h, plan._h, _ptr(in_cts), int(in_cts.shape[0]),
                                                _ptr(out), info["n_out"], ctypes.byref(lvl),
                                                ctypes.byref(sc)))
    else:
        _check(ctx, _lib().lib.fg_gcn_layer_axw_seeded(ctx._h, keys._h, plan._h, _ptr(in_cts),
                                                       int(in_cts.shape[0]), int(seed), _ptr(out),
                                                       info["n_out"], ctypes.byref(lvl), ctypes.byref(sc)))
    return out, lvl.value, sc.value


def gcn_layer_batch(ctx, keys, plans, ins, outs, streams=0, graph=True, tune=False, seeds=None):
    """Several layers at once (inputs on the device or in page-locked host
    memory, outputs on the device): query q runs plans[q] on ins[q] into
    outs[q]; tune picks the kernels' launch configuration by timing on the
    first call.  With seeds given, ins[q] are the c0 parts of seeded
    ciphertexts of seeds[q].  Returns (output levels, streams used)."""
    nat = _lib()
    n = len(plans)
    assert len(ins) == n and len(outs) == n
    P = (ctypes.c_void_p * n)(*[p._h.value if isinstance(p._h, ctypes.c_void_p) else p._h for p in plans])
    I = (ctypes.c_void_p * n)(*[_ptr(x).value for x in ins])
    O = (ctypes.c_void_p * n)(*[_ptr(x).value for x in outs])
    lv = (ctypes.c_int * n)()
    su = ctypes.c_int()
    o = nat.BatchOpts(int(streams), 1 if graph else 0, 1 if tune else 0)
    if seeds is None:
        _check(ctx, nat.lib.fg_gcn_layer_batch(ctx._h, keys._h, P, n, I, O, ctypes.byref(o), lv,
                                               ctypes.byref(su)))
    else:
        assert len(seeds) == n
        S = (ctypes.c_uint64 * n)(*[int(v) for v in seeds])
        _check(ctx, nat.lib.fg_gcn_layer_batch_seeded(ctx._h, keys._h, P, n, I, S, O, ctypes.byref(o), lv,
                                                      ctypes.byref(su)))
    return list(lv), su.value


TUNING_FIELDS = ("ntt_cols", "ntt_rows", "ntt_tw", "ks_split", "ks_cols", "modup_fused", "moddown_fused",
                 "gmac_groups", "gmac_regs", "kara")


def batch_tuning(ctx):
    """({field: value for each of TUNING_FIELDS}, [ms of each configuration
    tried, the default first])."""
    cfg = (ctypes.c_int * len(TUNING_FIELDS))()
    ms = np.zeros(64, np.float64)
    n = ctypes.c_int()
    _check(ctx, _lib().lib.fg_batch_tuning(ctx._h, cfg, ctypes.c_void_p(ms.ctypes.data), 64, ctypes.byref(n)))
    return dict(zip(TUNING_FIELDS, list(cfg))), [float(v) for v in ms[:n.value]]


def set_tuning(ctx, ntt_cols=8, ntt_rows=8, ntt_tw=0, ks_split=0, ks_cols=1, modup_fused=1,
               moddown_fused=0, gmac_groups=7, gmac_regs=1, kara=1):
    """Fix the launch configuration of the context's later calls."""
    cfg = (ctypes.c_int * len(TUNING_FIELDS))(ntt_cols, ntt_rows, ntt_tw, ks_split, ks_cols, modup_fused,
                                              moddown_fused, gmac_groups, gmac_regs, kara)
    _check(ctx, _lib().lib.fg_ctx_set_tuning(ctx._h, cfg))


N_PLAN_FEATURES = 15


def plan_features(params, row_ptr, col, val, W, perm, t=0, radix_bits=0, aoo=True, min_out_level=0,
                  n_sampled=0, in_level=0):
    """The learned planner's statistics of one candidate plan (host only)."""
    nat = _lib()
    q_bits, p_bits = params["q_bits"], params["p_bits"]
    qb = (ctypes.c_int * len(q_bits))(*q_bits)
    pb = (ctypes.c_int * len(p_bits))(*p_bits)
    prm = nat.Params(params["log_n"], len(q_bits), qb, len(p_bits), pb, params["alpha"],
                     float(params["log_scale"]))
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    F, Fp = W.shape
    o = nat.PlanOpts(int(t), int(radix_bits), 1 if aoo else 0, int(min_out_level), int(n_sampled),
                     int(in_level), 0)
    out = np.zeros(N_PLAN_FEATURES, np.float32)
    rc = nat.lib.fg_plan_features(ctypes.byref(prm), ctypes.c_void_p(row_ptr.ctypes.data),
                                  ctypes.c_void_p(col.ctypes.data), ctypes.c_void_p(val.ctypes.data),
                                  row_ptr.size - 1, ctypes.c_void_p(W.ctypes.data), F, Fp,
                                  ctypes.c_void_p(perm.ctypes.data), ctypes.byref(o),
                                  ctypes.c_void_p(out.ctypes.data))
    if rc != 0:
        raise FicgcnError(rc, "plan features failed")
    return out


INT_MUL_OPS = {"mad.wide.u32": 0, "mul.hi.u32": 1, "mad.lo.u32": 2, "mad.cc.pair": 3}


def int_mul_peak(ctx, op="mad.wide.u32"):
    """Measured rate (operations per second, whole GPU) of one 32-bit
    multiply form (INT_MUL_OPS; "mad.cc.pair" = a 32 x 32 -> 64-bit product
    added to a 64-bit sum by a carry-chained pair, the step of the split
    products): the ALU roof of the modular kernels."""
    r = ctypes.c_double()
    _check(ctx, _lib().lib.fg_int_mul_peak(ctx._h, INT_MUL_OPS[op], ctypes.byref(r)))
    return r.value


MODE_SPINTRA, MODE_INTER = 0, 1


def select_mode(params, row_ptr, col, val, W, perm, layer, n_copies, lat=(20.0, 1.0, 1.0),
                max_inter_cts=0.0, t=0, radix_bits=0, aoo=True, min_out_level=0, n_sampled=0,
                in_level=0):
    """Aggregation mode of one layer (host only): (mode, {"spintra": cost,
    "inter": cost}, {"rotations", "terms", "inter_inputs", "log_t"}).
    lat = (L_rot, L_pmult, L_add)."""
    nat = _lib()
    q_bits, p_bits = params["q_bits"], params["p_bits"]
    qb = (ctypes.c_int * len(q_bits))(*q_bits)
    pb = (ctypes.c_int * len(p_bits))(*p_bits)
    prm = nat.Params(params["log_n"], len(q_bits), qb, len(p_bits), pb, params["alpha"],
                     float(params["log_scale"]))
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    F, Fp = W.shape
    o = nat.PlanOpts(int(t), int(radix_bits), 1 if aoo else 0, int(min_out_level), int(n_sampled),
                     int(in_level), 0)
    la = np.ascontiguousarray(lat, dtype=np.float64)
    mode = ctypes.c_int()
    cost = np.zeros(2, np.float64)
    cnt = np.zeros(4, np.int64)
    rc = nat.lib.fg_select_mode(ctypes.byref(prm), ctypes.c_void_p(row_ptr.ctypes.data),
                                ctypes.c_void_p(col.ctypes.data), ctypes.c_void_p(val.ctypes.data),
                                row_ptr.size - 1, ctypes.c_void_p(W.ctypes.data), F, Fp,
                                ctypes.c_void_p(perm.ctypes.data), ctypes.byref(o), int(layer),
                                int(n_copies), ctypes.c_void_p(la.ctypes.data), float(max_inter_cts),
                                ctypes.byref(mode), ctypes.c_void_p(cost.ctypes.data),
                                ctypes.c_void_p(cnt.ctypes.data))
    if rc != 0:
        raise FicgcnError(rc, "mode selection failed")
    return (mode.value, {"spintra": float(cost[0]), "inter": float(cost[1])},
            {"rotations": int(cnt[0]), "terms": int(cnt[1]), "inter_inputs": int(cnt[2]),
             "log_t": int(cnt[3])})


class Mlp:
    """The learned planner's latency model on the GPU (fg_mlp_*)."""

    def __init__(self, n_in, hidden, params):
        nat = _lib()
        self.n_in, self.hidden = int(n_in), int(hidden)
        p = np.ascontiguousarray(params, dtype=np.float32)
        h = ctypes.c_void_p()
        rc = nat.lib.fg_mlp_create(self.n_in, self.hidden, ctypes.c_void_p(p.ctypes.data), ctypes.byref(h))
        if rc != 0:
            raise FicgcnError(rc, (nat.lib.fg_last_error(None) or b"").decode())
        self._h = h
        self.n_params = p.size

    def _rc(self, rc):
        if rc != 0:
            raise FicgcnError(rc, (_lib().lib.fg_last_error(None) or b"").decode())

    def params(self):
        out = np.zeros(self.n_params, np.float32)
        self._rc(_lib().lib.fg_mlp_params(self._h, ctypes.c_void_p(out.ctypes.data)))
        return out

    def forward(self, X):
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.zeros(X.shape[0], np.float32)
        self._rc(_lib().lib.fg_mlp_forward(self._h, ctypes.c_void_p(X.ctypes.data), X.shape[0],
                                            ctypes.c_void_p(y.ctypes.data)))
        return y

    def grad(self, X, y):
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        loss = ctypes.c_float()
        g = np.zeros(self.n_params, np.float32)
        self._rc(_lib().lib.fg_mlp_grad(self._h, ctypes.c_void_p(X.ctypes.data),
                                         ctypes.c_void_p(y.ctypes.data), X.shape[0], ctypes.byref(loss),
                                         ctypes.c_void_p(g.ctypes.data)))
        return loss.value, g

    def train(self, X, y, steps, lr):
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        losses = np.zeros(max(1, steps), np.float32)
        self._rc(_lib().lib.fg_mlp_train(self._h, ctypes.c_void_p(X.ctypes.data),
                                          ctypes.c_void_p(y.ctypes.data), X.shape[0], int(steps),
                                          ctypes.c_float(lr), ctypes.c_void_p(losses.ctypes.data)))
        return losses[:steps]

    def choose(self, features):
        F = np.ascontiguousarray(features, dtype=np.float32)
        pred = np.zeros(F.shape[0], np.float32)
        best = ctypes.c_int()
        self._rc(_lib().lib.fg_plan_choose(self._h, ctypes.c_void_p(F.ctypes.data), F.shape[0],
                                            ctypes.c_void_p(pred.ctypes.data), ctypes.byref(best)))
        return best.value, pred

    def close(self):
        if self._h is not None:
            _lib().lib.fg_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mul_relin_rescale(ctx, keys, a, b, level, out=None):
    """CMult of each pair: a, b [n][2][level+1][N] (or [2][level+1][N]) ->
    [n][2][level][N]; b may be a itself (the x^2 activation)."""
    single = len(a.shape) == 3
    n = 1 if single else int(a.shape[0])
    if out is None:
        out = _like(a, (2, level, ctx.n) if single else (n, 2, level, ctx.n))
    _check(ctx, _lib().lib.fg_mul_relin_rescale(ctx._h, keys._h, _ptr(a), _ptr(b), n, int(level),
                                                _ptr(out)))
    return out


def rotate(ctx, keys, ct, level, k, out=None):
    if out is None:
        out = _like(ct, (2, level + 1, ctx.n))
    _check(ctx, _lib().lib.fg_rotate(ctx._h, keys._h, _ptr(ct), level, int(k), _ptr(out)))
    return out


def rescale(ctx, ct, level, out=None):
    if out is None:
        out = _like(ct, (2, level, ctx.n))
    _check(ctx, _lib().lib.fg_rescale(ctx._h, _ptr(ct), level, _ptr(out)))
    return out


def poly_mul(ctx, a, b, level, out=None):
    if out is None:
        out = _like(a, (level + 1, ctx.n))
    _check(ctx, _lib().lib.fg_poly_mul(ctx._h, _ptr(a), _ptr(b), level, _ptr(out)))
    return out


def ntt(ctx, data, prime_idx, inverse=False):
    """In-place NTT of a CUDA tensor [count][N]; limb c uses prime prime_idx[c % len]."""
    pid = (ctypes.c_int * len(prime_idx))(*prime_idx)
    count = data.numel() // ctx.n
    _check(ctx, _lib().lib.fg_ntt(ctx._h, _ptr(data), count, pid, len(prime_idx), 1 if inverse else 0))
    return data
