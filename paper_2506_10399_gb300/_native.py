"""ctypes loader of libficgcn.so (the C ABI of include/ficgcn.h).

The library must be built in-tree (build.py); importing this module without
it raises ImportError -- there is no fallback implementation.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libficgcn.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libficgcn.so is missing: build it with paper_2506_10399_gb300/build.py "
                      "(or __graft_entry__.build()); there is no CPU fallback")

lib = ctypes.CDLL(LIB_PATH)

c_int, c_u64, c_size, c_double = ctypes.c_int, ctypes.c_uint64, ctypes.c_size_t, ctypes.c_double
c_void_p = ctypes.c_void_p
P = ctypes.POINTER


class Params(ctypes.Structure):
    _fields_ = [("log_n", c_int), ("n_q", c_int), ("q_bits", P(c_int)), ("n_p", c_int),
                ("p_bits", P(c_int)), ("alpha", c_int), ("log_scale", c_double)]


class PlanOpts(ctypes.Structure):
    _fields_ = [("t", c_int), ("radix_bits", c_int), ("aoo", c_int), ("min_out_level", c_int),
                ("n_sampled", c_int), ("in_level", c_int), ("no_encode", c_int)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("streams", c_int), ("graph", c_int), ("tune", c_int)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("t", c_int), ("B", c_int), ("n_in", c_int), ("n_out", c_int), ("in_level", c_int),
                ("out_level", c_int), ("n_groups", c_int), ("n_masks", c_int), ("n_keys", c_int),
                ("rotations", ctypes.c_int64), ("masked_products", ctypes.c_int64)]


SIGS = {
    "fg_ctx_create": (c_int, [P(Params), c_void_p, P(c_void_p)]),
    "fg_ctx_destroy": (c_int, [c_void_p]),
    "fg_last_error": (ctypes.c_char_p, [c_void_p]),
    "fg_ctx_primes": (c_int, [c_void_p, c_void_p, c_void_p]),
    "fg_ctx_device_bytes": (c_int, [c_void_p, P(c_size)]),
    "fg_free": (None, [c_void_p]),
    "fg_ctx_time_kernels": (c_int, [c_void_p, ctypes.c_char_p]),
    "fg_ctx_kernel_times": (c_int, [c_void_p, P(c_double), P(ctypes.c_int64), P(c_double)]),
    "fg_ctx_launch_count": (c_int, [c_void_p, P(ctypes.c_int64)]),
    "fg_keygen": (c_int, [c_void_p, c_u64, P(ctypes.c_int32), c_int, c_int, P(c_void_p), P(c_size),
                          P(c_void_p), P(c_size)]),
    "fg_encode_plain": (c_int, [c_void_p, c_void_p, c_int, c_double, c_int, c_void_p]),
    "fg_encrypt": (c_int, [c_void_p, c_void_p, c_size, c_u64, c_u64, c_void_p, c_int, c_void_p]),
    "fg_pack_features": (c_int, [c_void_p, c_void_p, c_size, c_u64, c_void_p, c_int, c_int,
                                 c_void_p, c_int, c_void_p, P(c_int)]),
    "fg_pack_features_seeded": (c_int, [c_void_p, c_void_p, c_size, c_u64, c_void_p, c_int, c_int,
                                        c_void_p, c_int, c_void_p, P(c_int)]),
    "fg_expand_seeded": (c_int, [c_void_p, c_u64, c_void_p, c_int, c_int, c_void_p]),
    "fg_decrypt": (c_int, [c_void_p, c_void_p, c_size, c_void_p, c_int, c_void_p]),
    "fg_pack_neighbor_copies": (c_int, [c_void_p, c_void_p, c_size, ctypes.c_uint64, c_void_p, c_int,
                                        c_int, c_void_p, c_int, c_void_p, c_void_p]),
    "fg_decrypt_decode": (c_int, [c_void_p, c_void_p, c_size, c_void_p, c_int, c_double, c_void_p]),
    "fg_load_evk": (c_int, [c_void_p, c_void_p, c_size, P(c_void_p)]),
    "fg_keys_destroy": (c_int, [c_void_p]),
    "fg_keys_export": (c_int, [c_void_p, ctypes.c_int32, c_int, c_void_p, c_void_p]),
    "fg_plan_build": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_int,
                              c_int, c_void_p, P(PlanOpts), P(c_void_p)]),
    "fg_plan_destroy": (c_int, [c_void_p]),
    "fg_plan_info": (c_int, [c_void_p, P(PlanInfo)]),
    "fg_plan_rotation_amounts": (c_int, [c_void_p, c_void_p, c_int, P(c_int)]),
    "fg_plan_describe": (c_int, [c_void_p, c_void_p, c_size, P(c_size)]),
    "fg_plan_set_plaintext": (c_int, [c_void_p, c_int, c_void_p]),
    "fg_plan_dry_run": (c_int, [P(Params), c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_int, c_int,
                                c_void_p, P(PlanOpts), c_void_p, c_size, P(c_size)]),
    "fg_node_order": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p, P(c_int)]),
    "fg_node_order_ex": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_void_p, P(c_int)]),
    "fg_plan_build_inter": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_void_p, c_int, c_int,
                                    c_void_p, P(PlanOpts), P(c_void_p)]),
    "fg_plan_features": (c_int, [P(Params), c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_int, c_int,
                                 c_void_p, P(PlanOpts), c_void_p]),
    "fg_plan_features_built": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "fg_select_mode": (c_int, [P(Params), c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_int, c_int,
                               c_void_p, P(PlanOpts), c_int, c_int, c_void_p, c_double, P(c_int),
                               c_void_p, c_void_p]),
    "fg_mlp_create": (c_int, [c_int, c_int, c_void_p, P(c_void_p)]),
    "fg_mlp_destroy": (c_int, [c_void_p]),
    "fg_mlp_params": (c_int, [c_void_p, c_void_p]),
    "fg_mlp_forward": (c_int, [c_void_p, c_void_p, c_int, c_void_p]),
    "fg_mlp_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
    "fg_mlp_train": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, ctypes.c_float, c_void_p]),
    "fg_plan_choose": (c_int, [c_void_p, c_void_p, c_int, c_void_p, P(c_int)]),
    "fg_mul_relin_rescale": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "fg_gcn_layer_batch": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p,
                                   P(BatchOpts), c_void_p, P(c_int)]),
    "fg_gcn_layer_batch_seeded": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p,
                                          P(BatchOpts), c_void_p, P(c_int)]),
    "fg_ctx_set_tuning": (c_int, [c_void_p, c_void_p]),
    "fg_ctx_release_workspace": (c_int, [c_void_p]),
    "fg_batch_tuning": (c_int, [c_void_p, c_void_p, c_void_p, c_int, P(c_int)]),
    "fg_gcn_layer_axw": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_int,
                                 P(c_int), P(c_double)]),
    "fg_gcn_layer_axw_seeded": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_u64, c_void_p,
                                        c_int, P(c_int), P(c_double)]),
    "fg_rotate": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "fg_rescale": (c_int, [c_void_p, c_void_p, c_int, c_void_p]),
    "fg_poly_mul": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    "fg_poly_mul_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    "fg_ntt": (c_int, [c_void_p, c_void_p, c_int, P(c_int), c_int, c_int]),
    "fg_int_mul_peak": (c_int, [c_void_p, c_int, P(c_double)]),
}

for _name, (_res, _args) in SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args

STATUS = {0: "FG_OK", -1: "FG_EINVAL", -2: "FG_ELEVEL", -3: "FG_EKEY", -4: "FG_ECUDA",
          -5: "FG_EOOM", -6: "FG_ETIMEOUT", -7: "FG_ENODEV"}
