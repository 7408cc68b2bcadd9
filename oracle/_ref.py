"""ctypes binding of the oracle's exact-integer core (ckks_ref.c).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Arrays are numpy
uint64 / int64, C-contiguous, limb-major ``[n_limbs][N]``.
"""
import ctypes

import numpy as np

from . import LIB_PATH, build

build()
_lib = ctypes.CDLL(LIB_PATH)

_u64 = ctypes.c_uint64
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_intp = ctypes.POINTER(ctypes.c_int)
_int = ctypes.c_int

_lib.ref_is_prime.argtypes = [_u64]
_lib.ref_is_prime.restype = _int
_lib.ref_gen_primes.argtypes = [_int, _int, _intp, _u64p]
_lib.ref_gen_primes.restype = _int
_lib.ref_find_psi.argtypes = [_int, _u64]
_lib.ref_find_psi.restype = _u64
_lib.ref_mulmod.argtypes = [_u64, _u64, _u64]
_lib.ref_mulmod.restype = _u64
_lib.ref_invmod.argtypes = [_u64, _u64]
_lib.ref_invmod.restype = _u64
_lib.ref_negacyclic_mul_schoolbook.argtypes = [_u64p, _u64p, _u64p, _int, _u64]
_lib.ref_negacyclic_mul.argtypes = [_u64p, _u64p, _u64p, _int, _u64, _u64]
_lib.ref_automorphism.argtypes = [_u64p, _u64p, _int, _u64, _u64]
_lib.ref_base_convert.argtypes = [_u64p, _int, _u64p, _u64p, _int, _u64p, _int]
_lib.ref_rescale.argtypes = [_u64p, _int, _u64p, _u64p, _int]
_lib.ref_moddown.argtypes = [_u64p, _int, _u64p, _int, _u64p, _u64p, _int]
_lib.ref_mul_scalar.argtypes = [_u64p, _u64, _u64p, _int, _u64]
_lib.ref_mac_scalar.argtypes = [_u64p, _u64, _u64p, _int, _u64]
_lib.ref_splitmix_first.argtypes = [_u64, _u64, _u64, _int, _u64p]
_lib.ref_splitmix_first.restype = _u64
_lib.ref_sample_ternary.argtypes = [_u64, _u64, _u64, _int, _i64p]
_lib.ref_sample_gauss.argtypes = [_u64, _u64, _u64, _int, _i64p]
_lib.ref_gauss_table.argtypes = [_u64p]
_lib.ref_sample_uniform.argtypes = [_u64, _u64, _u64, _u64p, _int, _int, _u64p]
_lib.ref_sample_uniform_wide.argtypes = [_u64, _u64, _u64, _u64p, _int, _int, _u64p]


def _p(a):
    return a.ctypes.data_as(_u64p)


def _pi(a):
    return a.ctypes.data_as(_i64p)


def _u(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def _arr(xs):
    return np.ascontiguousarray(np.array([int(x) for x in xs], dtype=np.uint64))


def is_prime(n):
    return bool(_lib.ref_is_prime(int(n)))


def gen_primes(log_n, bits):
    bits = list(bits)
    cb = (ctypes.c_int * len(bits))(*bits)
    out = np.zeros(len(bits), dtype=np.uint64)
    if _lib.ref_gen_primes(log_n, len(bits), cb, _p(out)) != 0:
        raise ValueError("no prime of the requested size")
    return [int(x) for x in out]


def find_psi(n, q):
    return int(_lib.ref_find_psi(n, int(q)))


def mulmod(a, b, q):
    return int(_lib.ref_mulmod(int(a), int(b), int(q)))


def invmod(a, q):
    return int(_lib.ref_invmod(int(a), int(q)))


def negacyclic_mul_schoolbook(a, b, q):
    a, b = _u(a), _u(b)
    c = np.zeros_like(a)
    _lib.ref_negacyclic_mul_schoolbook(_p(a), _p(b), _p(c), a.size, int(q))
    return c


def negacyclic_mul(a, b, q, psi):
    a, b = _u(a), _u(b)
    c = np.zeros_like(a)
    _lib.ref_negacyclic_mul(_p(a), _p(b), _p(c), a.size, int(q), int(psi))
    return c


def automorphism(a, g, q):
    a = _u(a)
    out = np.zeros_like(a)
    _lib.ref_automorphism(_p(a), _p(out), a.size, int(g), int(q))
    return out


def base_convert(x, b_primes, c_primes):
    x = _u(x)
    n = x.shape[-1]
    bp, cp = _arr(b_primes), _arr(c_primes)
    out = np.zeros((len(c_primes), n), dtype=np.uint64)
    _lib.ref_base_convert(_p(x), len(b_primes), _p(bp), _p(out), len(c_primes), _p(cp), n)
    return out


def rescale(c, primes):
    """c: [l+1][N] over primes[0..l]; returns [l][N]."""
    c = _u(c)
    nl, n = c.shape
    pr = _arr(primes[:nl])
    out = np.zeros((nl - 1, n), dtype=np.uint64)
    _lib.ref_rescale(_p(c), nl, _p(pr), _p(out), n)
    return out


def moddown(u, q_primes, p_primes):
    u = _u(u)
    n = u.shape[-1]
    qp, pp = _arr(q_primes), _arr(p_primes)
    out = np.zeros((len(q_primes), n), dtype=np.uint64)
    _lib.ref_moddown(_p(u), len(q_primes), _p(qp), len(p_primes), _p(pp), _p(out), n)
    return out


def mul_scalar(a, s, q):
    a = _u(a)
    out = np.zeros_like(a)
    _lib.ref_mul_scalar(_p(a), int(s) % int(q), _p(out), a.size, int(q))
    return out


def mac_scalar(a, s, out, q):
    """out += a*s mod q, in place (out must be a contiguous uint64 array)."""
    a = _u(a)
    assert out.flags["C_CONTIGUOUS"] and out.dtype == np.uint64
    _lib.ref_mac_scalar(_p(a), int(s) % int(q), _p(out), a.size, int(q))


def splitmix(seed, purpose, index, count):
    out = np.zeros(count, dtype=np.uint64)
    _lib.ref_splitmix_first(seed, purpose, index, count, _p(out))
    return out


def sample_ternary(seed, purpose, index, n):
    out = np.zeros(n, dtype=np.int64)
    _lib.ref_sample_ternary(seed, purpose, index, n, _pi(out))
    return out


def sample_gauss(seed, purpose, index, n):
    """Discrete Gaussian noise, sigma = 3.2, |x| <= 19 (see ckks_ref.c)."""
    out = np.zeros(n, dtype=np.int64)
    _lib.ref_sample_gauss(seed, purpose, index, n, _pi(out))
    return out


def gauss_table():
    out = np.zeros(20, dtype=np.uint64)
    _lib.ref_gauss_table(_p(out))
    return [int(v) for v in out]


def sample_uniform(seed, purpose, index, primes, n):
    pr = _arr(primes)
    out = np.zeros((len(primes), n), dtype=np.uint64)
    _lib.ref_sample_uniform(seed, purpose, index, _p(pr), len(primes), n, _p(out))
    return out


def sample_uniform_wide(seed, purpose, index, primes, n):
    """Uniform residues [len(primes)][n], each from two stream words,
    (w_hi 2^64 + w_lo) mod q, no rejection (see ckks_ref.c)."""
    pr = _arr(primes)
    out = np.zeros((len(primes), n), dtype=np.uint64)
    _lib.ref_sample_uniform_wide(seed, purpose, index, _p(pr), len(primes), n, _p(out))
    return out
