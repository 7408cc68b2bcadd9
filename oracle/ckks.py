"""CKKS-RNS primitives of the oracle.  TEST INFRASTRUCTURE ONLY.

Everything here follows the CKKS preliminaries of the paper (Sec. 2.1):
ciphertexts c in R_Q^2 decrypt as c0 + c1*s = m + e (mod Q), Q = prod q_i,
the ring is Z_Q[X]/(X^N+1), a ciphertext holds N/2 slots, and
Rot(Enc(v_0..v_{N/2-1}), k) = Enc(v_k, .., v_{N/2-1}, v_0, .., v_{k-1}).
What the paper leaves to the CKKS literature (RNS moduli, hybrid key
switching, rescale rounding, sampling) is written here in the reading the
library implements too; each reading is named at its function.

Representation: a plaintext or one ciphertext part at level l is uint64
[l+1][N] over q_0..q_l, coefficient domain, residues in [0, q).  A
ciphertext is uint64 [2][l+1][N].  Extended-basis polynomials (after ModUp)
are [l+1+K][N] over q_0..q_l, p_0..p_{K-1}.
"""
import math

import numpy as np

from . import _ref

# purposes of the seeded streams (see ckks_ref.c, SplitMix64)
PURPOSE_SECRET = 1
PURPOSE_KEY_A = 2
PURPOSE_KEY_E = 3
PURPOSE_ENC_A = 4
PURPOSE_ENC_E = 5
PURPOSE_ENC_A_SEEDED = 6


class Params:
    """RNS-CKKS parameters.

    q_bits: bit sizes of q_0..q_L (q_0 first); p_bits: special primes;
    alpha: primes per key-switching digit; log_scale: log2 of Delta.
    Primes: for each size in the order q_bits then p_bits, the largest prime
    below 2^b that is 1 mod 2N and not taken yet.
    """

    def __init__(self, log_n, q_bits, p_bits, alpha, log_scale):
        self.log_n = int(log_n)
        self.n = 1 << self.log_n
        self.slots = self.n // 2
        primes = _ref.gen_primes(self.log_n, list(q_bits) + list(p_bits))
        self.q = primes[:len(q_bits)]
        self.p = primes[len(q_bits):]
        self.L = len(self.q) - 1
        self.K = len(self.p)
        self.alpha = int(alpha)
        self.log_scale = log_scale
        self.scale = float(2.0 ** log_scale)
        self._psi = {}

    def psi(self, prime):
        if prime not in self._psi:
            self._psi[prime] = _ref.find_psi(self.n, prime)
        return self._psi[prime]

    def ext_primes(self, level):
        return self.q[:level + 1] + self.p

    def key_limb(self, level, i):
        """Index, in a key generated over q_0..q_L, p.., of extended limb i at level l."""
        return i if i <= level else self.L + 1 + (i - level - 1)

    def digits(self, level):
        """Key-switching digits at level l: consecutive alpha primes of q_0..q_l."""
        return [list(range(j * self.alpha, min((j + 1) * self.alpha, level + 1)))
                for j in range(-(-(level + 1) // self.alpha))]

    def galois(self, k):
        """Galois element of a left rotation by k slots: 5^(k mod N/2) mod 2N."""
        return pow(5, int(k) % self.slots, 2 * self.n)

    def p_mod(self, prime):
        r = 1
        for pk in self.p:
            r = r * pk % prime
        return r


# ----------------------------------------------------------------------
# encoding (FP64, canonical embedding)
# ----------------------------------------------------------------------

def round_half_away(x):
    """Round to nearest, ties away from zero, for every float64 (as C round())."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    f = np.floor(a)                        # a - f is exact in FP64
    return np.sign(x) * (f + (a - f >= 0.5))


def _slot_exponents(params):
    two_n = 2 * params.n
    e = np.empty(params.slots, dtype=np.int64)
    v = 1
    for j in range(params.slots):
        e[j] = v
        v = v * 5 % two_n
    return e


def embed_inverse(params, z):
    """Real coefficients m with m(zeta^(5^j)) = z_j, zeta = exp(i pi / N).

    The N evaluation points zeta^e, e odd, are the slots (e = 5^j) and their
    conjugates (e = -5^j); m_i = (1/N) sum_e m(zeta^e) zeta^(-e i), which is
    the length-2N DFT of the point values placed at index e."""
    n = params.n
    z = np.zeros(params.slots, dtype=np.complex128) + np.asarray(z, dtype=np.complex128)
    e = _slot_exponents(params)
    v = np.zeros(2 * n, dtype=np.complex128)
    v[e] = z
    v[(2 * n - e) % (2 * n)] = np.conj(z)
    return np.fft.fft(v)[:n].real / n


def encode(params, z, scale, level, extended=False):
    """Plaintext [level+1][N]: round_half_away(scale * embed_inverse(z)) mod q_i;
    with extended=True also the residues mod p_0..p_{K-1} ([level+1+K][N]),
    for products taken in the key-switching basis."""
    m = round_half_away(scale * embed_inverse(params, z))
    primes = params.ext_primes(level) if extended else params.q[:level + 1]
    out = np.empty((len(primes), params.n), dtype=np.uint64)
    if np.max(np.abs(m)) < 2.0 ** 62:
        # every coefficient is an integer-valued double below 2^62: exact as
        # int64, and np.mod with a positive modulus returns [0, q)
        mi = m.astype(np.int64)
        for i, q in enumerate(primes):
            out[i] = np.mod(mi, np.int64(q)).astype(np.uint64)
        return out
    ints = [int(v) for v in m]
    for i, q in enumerate(primes):
        out[i] = np.array([v % q for v in ints], dtype=np.uint64)
    return out


def crt_centered(params, res):
    """CRT-lift residues [l+1][N] (over q_0..q_l) to Python ints in (-Q/2, Q/2]."""
    nl = res.shape[0]
    qs = params.q[:nl]
    Q = 1
    for q in qs:
        Q *= q
    acc = np.zeros(res.shape[1], dtype=object)
    for i, q in enumerate(qs):
        hat = Q // q
        coef = hat * pow(hat % q, -1, q)
        acc = acc + res[i].astype(object) * coef
    acc = acc % Q
    return np.where(acc > Q // 2, acc - Q, acc)


def decode(params, pt, scale):
    """Slots z_j = m(zeta^(5^j)) / scale of a plaintext given by its residues."""
    n = params.n
    m = crt_centered(params, pt)
    mf = np.array([float(v) for v in m], dtype=np.float64) / scale
    u = np.zeros(2 * n, dtype=np.complex128)
    u[:n] = mf
    w = np.fft.ifft(u) * (2 * n)           # w[e] = sum_i m_i zeta^(e i)
    return w[_slot_exponents(params)]


# ----------------------------------------------------------------------
# small integer polynomials
# ----------------------------------------------------------------------

def small_to_res(e, primes):
    """Signed small-integer coefficients -> residues [len(primes)][N]."""
    e = np.asarray(e, dtype=np.int64)
    return np.stack([np.where(e < 0, e + np.int64(q), e).astype(np.uint64) for q in primes])


def automorphism_small(e, g, n):
    """a(X) -> a(X^g) on signed integer coefficients."""
    out = np.zeros(n, dtype=np.int64)
    for i in range(n):
        t = i * g % (2 * n)
        if t < n:
            out[t] = e[i]
        else:
            out[t - n] = -e[i]
    return out


def poly_mul(params, a, b, primes):
    """Negacyclic product, limb by limb."""
    return np.stack([_ref.negacyclic_mul(a[i], b[i], q, params.psi(q))
                     for i, q in enumerate(primes)])


def add_res(a, b, primes):
    out = np.empty_like(a)
    for i, q in enumerate(primes):
        s = a[i] + b[i]
        out[i] = np.where(s >= np.uint64(q), s - np.uint64(q), s)
    return out


def sub_res(a, b, primes):
    out = np.empty_like(a)
    for i, q in enumerate(primes):
        out[i] = np.where(a[i] >= b[i], a[i] - b[i], a[i] + (np.uint64(q) - b[i]))
    return out


def neg_res(a, primes):
    out = np.empty_like(a)
    for i, q in enumerate(primes):
        out[i] = np.where(a[i] == 0, a[i], np.uint64(q) - a[i])
    return out


# ----------------------------------------------------------------------
# keys, encryption, decryption
# ----------------------------------------------------------------------

def keygen_secret(params, seed):
    """Ternary secret s: one SplitMix64 stream (seed, 1, 0)."""
    return _ref.sample_ternary(seed, PURPOSE_SECRET, 0, params.n)


def keygen_switch(params, seed, s, s_from, index):
    """Hybrid key-switching key from s_from to s (Han-Ki with alpha primes per
    digit), generated over q_0..q_L, p_0..p_{K-1}.  For each top-level digit
    D_j: a_j uniform, e_j noise,
      b_j = -a_j*s + e_j + P * [i in D_j] * s_from   (mod each q_i),
      b_j = -a_j*s + e_j                             (mod each p_k),
    i.e. the gadget P * (Q/D_j) * [(Q/D_j)^-1]_{D_j}, which is P mod the
    primes of D_j and 0 mod every other prime.  Streams: a from
    (seed, 2, index<<8 | j), e from (seed, 3, index<<8 | j).
    Returns a list over digits of (b, a), each [L+1+K][N]."""
    n = params.n
    primes = params.q + params.p
    s_res = small_to_res(s, primes)
    sf_res = small_to_res(s_from, primes)
    key = []
    for j, dig in enumerate(params.digits(params.L)):
        idx = (int(index) << 8) | j
        a = _ref.sample_uniform(seed, PURPOSE_KEY_A, idx, primes, n)
        e = _ref.sample_gauss(seed, PURPOSE_KEY_E, idx, n)
        e_res = small_to_res(e, primes)
        b = neg_res(poly_mul(params, a, s_res, primes), primes)
        b = add_res(b, e_res, primes)
        for i in dig:
            q = primes[i]
            gad = _ref.mul_scalar(sf_res[i], params.p_mod(q), q)
            b[i] = add_res(b[i:i + 1], gad[None, :], [q])[0]
        key.append((b, a))
    return key


def keygen_rotation(params, seed, s, k):
    """Rotation key for a left rotation by k: switches phi_g(s) -> s, with
    g = 5^k mod 2N; the key stream index is g."""
    g = params.galois(k)
    return keygen_switch(params, seed, s, automorphism_small(s, g, params.n), g)


def secret_square(params, s):
    """s^2 in R = Z[X]/(X^N+1) as integers (|coefficient| <= N): the
    negacyclic product mod q_0, read as a centred integer."""
    q = params.q[0]
    r = small_to_res(s, [q])[0]
    sq = _ref.negacyclic_mul(r, r, q, params.psi(q))
    return np.where(sq > q // 2, sq.astype(object) - q, sq.astype(object)).astype(np.int64)


def keygen_relin(params, seed, s):
    """Relinearisation key: switches s^2 -> s (the key of Sec. 2.1's CMult),
    the same hybrid construction as a rotation key with stream index 0 (no
    rotation key uses 0: Galois elements are odd)."""
    return keygen_switch(params, seed, s, secret_square(params, s), 0)


def mul_ct(params, a, b):
    """Tensor product of two ciphertexts at one level:
    (d0, d1, d2) = (a0 b0, a0 b1 + a1 b0, a1 b1), so that
    d0 + d1 s + d2 s^2 = (a0 + a1 s)(b0 + b1 s)."""
    nl = a.shape[1]
    primes = params.q[:nl]
    d0 = poly_mul(params, a[0], b[0], primes)
    d1 = add_res(poly_mul(params, a[0], b[1], primes), poly_mul(params, a[1], b[0], primes), primes)
    d2 = poly_mul(params, a[1], b[1], primes)
    return d0, d1, d2


def relinearize(params, d0, d1, d2, key):
    """(d0, d1) + KS(d2) with the relinearisation key: ModUp of d2, inner
    product with the key's digits over q_0..q_l, p.., ModDown of both sums
    (hybrid key switching as in rotate, without an automorphism)."""
    level = d0.shape[0] - 1
    ext = params.ext_primes(level)
    digits = modup(params, d2, level)
    u0 = np.zeros((len(ext), params.n), dtype=np.uint64)
    u1 = np.zeros((len(ext), params.n), dtype=np.uint64)
    for j, dj in enumerate(digits):
        kb, ka = key[j]
        for i, pr in enumerate(ext):
            kl = params.key_limb(level, i)
            psi = params.psi(pr)
            t0 = _ref.negacyclic_mul(dj[i], kb[kl], pr, psi)
            t1 = _ref.negacyclic_mul(dj[i], ka[kl], pr, psi)
            u0[i] = add_res(u0[i:i + 1], t0[None], [pr])[0]
            u1[i] = add_res(u1[i:i + 1], t1[None], [pr])[0]
    qs = params.q[:level + 1]
    r0 = _ref.moddown(u0, qs, params.p)
    r1 = _ref.moddown(u1, qs, params.p)
    return np.stack([add_res(d0, r0, qs), add_res(d1, r1, qs)])


def mul_relin_rescale(params, a, b, key):
    """CMult (Sec. 2.1): tensor product, relinearisation, rescale by q_l.
    The scale becomes scale_a * scale_b / q_l."""
    return rescale_ct(params, relinearize(params, *mul_ct(params, a, b), key))


def encrypt(params, seed, index, pt, s, level):
    """Secret-key encryption c = (-a*s + m + e, a) over q_0..q_l.
    Streams: a from (seed, 4, index), e from (seed, 5, index)."""
    primes = params.q[:level + 1]
    a = _ref.sample_uniform(seed, PURPOSE_ENC_A, index, primes, params.n)
    e = small_to_res(_ref.sample_gauss(seed, PURPOSE_ENC_E, index, params.n), primes)
    c0 = neg_res(poly_mul(params, a, small_to_res(s, primes), primes), primes)
    c0 = add_res(add_res(c0, pt[:level + 1], primes), e, primes)
    return np.stack([c0, a])


def seeded_a(params, seed, index, level):
    """The uniform part of a seeded ciphertext: drawn coefficient by
    coefficient from the stream (seed, 6, index) over q_0..q_level, two
    words each (_ref.sample_uniform_wide), so the receiver can regenerate it
    from (seed, index) alone."""
    return _ref.sample_uniform_wide(seed, PURPOSE_ENC_A_SEEDED, index, params.q[:level + 1], params.n)


def encrypt_seeded(params, seed, index, pt, s, level):
    """Secret-key encryption with a regenerable uniform part (the seeded,
    compressed form of a symmetric ciphertext): c0 = -a*s + m + e with a =
    seeded_a(seed, index) and e from (seed, 5, index).  Only c0 (and the
    seed) travels; expand_seeded rebuilds (c0, a)."""
    primes = params.q[:level + 1]
    a = seeded_a(params, seed, index, level)
    e = small_to_res(_ref.sample_gauss(seed, PURPOSE_ENC_E, index, params.n), primes)
    c0 = neg_res(poly_mul(params, a, small_to_res(s, primes), primes), primes)
    return add_res(add_res(c0, pt[:level + 1], primes), e, primes)


def expand_seeded(params, seed, index, c0):
    """The full ciphertext (c0, a) of a seeded one."""
    return np.stack([c0, seeded_a(params, seed, index, c0.shape[0] - 1)])


def decrypt(params, ct, s):
    """m' = c0 + c1*s (mod q_i) at the ciphertext's level."""
    nl = ct.shape[1]
    primes = params.q[:nl]
    return add_res(ct[0], poly_mul(params, ct[1], small_to_res(s, primes), primes), primes)


# ----------------------------------------------------------------------
# evaluation
# ----------------------------------------------------------------------

def level_of(ct):
    return ct.shape[1] - 1


def add_ct(params, a, b):
    primes = params.q[:a.shape[1]]
    return np.stack([add_res(a[0], b[0], primes), add_res(a[1], b[1], primes)])


def drop_ct(ct):
    """Level drop without division: discard the top limb."""
    return np.ascontiguousarray(ct[:, :-1])


def rescale_ct(params, ct):
    """Divide by the top prime q_l, rounding to the nearest integer, both parts."""
    primes = params.q[:ct.shape[1]]
    return np.stack([_ref.rescale(ct[0], primes), _ref.rescale(ct[1], primes)])


def pmult(params, pt, ct):
    """Plaintext-ciphertext product m (x) c: both parts times the plaintext."""
    nl = ct.shape[1]
    primes = params.q[:nl]
    return np.stack([poly_mul(params, pt[:nl], ct[0], primes),
                     poly_mul(params, pt[:nl], ct[1], primes)])


def const_mac(params, acc, ct, c):
    """acc += c * ct for a signed integer constant c, reduced mod each q_i."""
    for part in range(2):
        for i in range(ct.shape[1]):
            q = params.q[i]
            _ref.mac_scalar(ct[part, i], int(c) % q, acc[part, i], q)


def modup(params, d, level):
    """ModUp of a level-l polynomial, one output per digit D_j: the digit's
    own limbs are kept, every other prime of q_0..q_l, p.. gets
    Conv_{D_j -> that prime}([d]_{D_j}) (approximate, no overflow fix)."""
    ext = params.ext_primes(level)
    out = []
    for dig in params.digits(level):
        lifted = np.empty((len(ext), params.n), dtype=np.uint64)
        others = [i for i in range(len(ext)) if i not in dig]
        conv = _ref.base_convert(d[dig], [params.q[i] for i in dig], [ext[i] for i in others])
        for r, i in enumerate(others):
            lifted[i] = conv[r]
        for i in dig:
            lifted[i] = d[i]
        out.append(lifted)
    return out


def keyswitch_ext(params, ct, k, key, digits=None):
    """The key-switching half of Rot(c, k) before ModDown: the inner product
    (u0, u1) = sum_j phi_g(ModUp_j(c1)) * key_j over q_0..q_l, p.. (hoisted
    digits as in rotate), and phi_g(c0) over q_0..q_l.  ModDown(u) +
    (phi_g(c0), 0) is Rot(c, k)."""
    level = level_of(ct)
    g = params.galois(k)
    ext = params.ext_primes(level)
    if digits is None:
        digits = modup(params, ct[1], level)
    u0 = np.zeros((len(ext), params.n), dtype=np.uint64)
    u1 = np.zeros((len(ext), params.n), dtype=np.uint64)
    for j, dj in enumerate(digits):
        kb, ka = key[j]
        for i, pr in enumerate(ext):
            dg = _ref.automorphism(dj[i], g, pr)
            kl = params.key_limb(level, i)
            psi = params.psi(pr)
            t0 = _ref.negacyclic_mul(dg, kb[kl], pr, psi)
            t1 = _ref.negacyclic_mul(dg, ka[kl], pr, psi)
            u0[i] = add_res(u0[i:i + 1], t0[None], [pr])[0]
            u1[i] = add_res(u1[i:i + 1], t1[None], [pr])[0]
    qs = params.q[:level + 1]
    c0g = np.stack([_ref.automorphism(ct[0, i], g, q) for i, q in enumerate(qs)])
    return np.stack([u0, u1]), c0g


def moddown_ct(params, u):
    """ModDown of both parts of an extended-basis pair [2][l+1+K][N]."""
    level = u.shape[1] - 1 - params.K
    qs = params.q[:level + 1]
    return np.stack([_ref.moddown(u[0], qs, params.p), _ref.moddown(u[1], qs, params.p)])


def rotate(params, ct, k, key, digits=None):
    """Rot(c, k) in the hoisted order: ModUp of c1 first (or the digits
    given, shared by every rotation of the same ciphertext), then the
    automorphism phi_g on each lifted digit, the inner product with the
    key's digits over q_0..q_l, p.., ModDown of both sums, and phi_g(c0)
    added to the first part.  The key is the full top-level key; limbs
    above l are skipped and only the level's digits are used."""
    level = level_of(ct)
    g = params.galois(k)
    ext = params.ext_primes(level)
    if digits is None:
        digits = modup(params, ct[1], level)
    u0 = np.zeros((len(ext), params.n), dtype=np.uint64)
    u1 = np.zeros((len(ext), params.n), dtype=np.uint64)
    for j, dj in enumerate(digits):
        kb, ka = key[j]
        for i, pr in enumerate(ext):
            dg = _ref.automorphism(dj[i], g, pr)
            kl = params.key_limb(level, i)
            psi = params.psi(pr)
            t0 = _ref.negacyclic_mul(dg, kb[kl], pr, psi)
            t1 = _ref.negacyclic_mul(dg, ka[kl], pr, psi)
            u0[i] = add_res(u0[i:i + 1], t0[None], [pr])[0]
            u1[i] = add_res(u1[i:i + 1], t1[None], [pr])[0]
    qs = params.q[:level + 1]
    r0 = _ref.moddown(u0, qs, params.p)
    r1 = _ref.moddown(u1, qs, params.p)
    c0g = np.stack([_ref.automorphism(ct[0, i], g, q) for i, q in enumerate(qs)])
    return np.stack([add_res(c0g, r0, qs), r1])
