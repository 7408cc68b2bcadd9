"""Reference CPU CKKS-RNS evaluator of one encrypted GCN layer.

TEST INFRASTRUCTURE ONLY.  This package is the oracle the CUDA library is
checked against: plain, slow, exact integer arithmetic (``ckks_ref.c``) plus
FP64 encoding and the SpIntra-CA planner written from the paper's text.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the library and never
imports it.

Modules
  _ref      ctypes binding of the exact-integer core (ckks_ref.c)
  ckks      parameters, encode/decode, keys, encryption, rotation, rescale
  planner   latency-aware packing, AOO shifts, SpIntra-CA lanes and masks
  layer     the encrypted A.X.W layer executed step by step on a plan, in
            the paper's step order and in the double-hoisted form
  noo       node order optimisation (Alg. 1)
  mlp       the learned planner's latency model in FP64

Parity status: every function is pinned by tests/test_oracle_*.py and
tests/test_noo.py; the NOO heuristic's output (a node order) is an input to
parity, never a parity target.
"""
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libckks_ref.so")


def build(force=False):
    """Compile ckks_ref.c into libckks_ref.so beside it (plain gcc, -O2)."""
    src = os.path.join(_HERE, "ckks_ref.c")
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= os.path.getmtime(src)):
        return LIB_PATH
    tmp = LIB_PATH + ".tmp.%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, LIB_PATH)
    return LIB_PATH
