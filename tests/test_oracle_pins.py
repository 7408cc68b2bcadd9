"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: Python
big-integer arithmetic, closed forms, ring identities, the paper's stated
examples (tests/golden/paper_examples.json), or the FP64 product A-hat X W.
A plausible slip anywhere (a dropped term, a wrong sign or index, a
transposed operand) fails at least one of them; test_planted_mistakes shows
that for a few such slips.
"""
import json
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

from oracle import _ref, ckks, layer, planner
from paper_2506_10399_gb300 import workloads as wl

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))


# ---------------------------------------------------------------- helpers
def py_is_prime(n):
    """Independent check: Miller-Rabin with 40 random witnesses (Python ints)."""
    if n < 4:
        return n in (2, 3)
    if n % 2 == 0:
        return False
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    rnd = random.Random(n)
    for _ in range(40):
        a = rnd.randrange(2, n - 1)
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def py_negacyclic(a, b, q):
    n = len(a)
    c = [0] * n
    for i in range(n):
        for j in range(n):
            k = i + j
            if k < n:
                c[k] += int(a[i]) * int(b[j])
            else:
                c[k - n] -= int(a[i]) * int(b[j])
    return [x % q for x in c]


def crt(residues, primes):
    Q = 1
    for p in primes:
        Q *= p
    x = 0
    for r, p in zip(residues, primes):
        h = Q // p
        x += int(r) * h * pow(h % p, -1, p)
    return x % Q, Q


def rand_res(rng, primes, n):
    return np.stack([np.array([rng.randrange(q) for _ in range(n)], dtype=np.uint64)
                     for q in primes])


def small_params(log_n=10, nq=4, qb=40, npr=1, alpha=1, log_scale=40):
    return ckks.Params(log_n, [60] + [qb] * (nq - 1), [60] * npr, alpha, log_scale)


# ---------------------------------------------------------------- primes
@pytest.mark.parametrize("log_n,bits", [(4, [20, 20, 18]), (12, [60, 40, 40, 60]),
                                        (16, [60, 45, 45, 60])])
def test_primes_largest_ntt_friendly(log_n, bits):
    ps = _ref.gen_primes(log_n, bits)
    two_n = 2 << log_n
    for i, (p, b) in enumerate(zip(ps, bits)):
        assert py_is_prime(p) and p % two_n == 1 and p < (1 << b)
        assert p not in ps[:i]
        # no larger unused candidate below 2^b is prime
        c = (1 << b) - two_n + 1
        while c > p:
            if c not in ps[:i]:
                assert not py_is_prime(c)
            c -= two_n


def test_is_prime_small_numbers():
    small = [n for n in range(2, 2000) if all(n % d for d in range(2, int(n ** 0.5) + 1))]
    assert [n for n in range(2000) if _ref.is_prime(n)] == small
    assert _ref.is_prime((1 << 61) - 1) and not _ref.is_prime(((1 << 31) - 1) * ((1 << 31) + 11))


# ---------------------------------------------------------------- products
@pytest.mark.parametrize("n", [4, 8, 16])
def test_schoolbook_vs_bigint(n):
    q = _ref.gen_primes(int(math.log2(n)), [30])[0]
    rng = random.Random(n)
    a = [rng.randrange(q) for _ in range(n)]
    b = [rng.randrange(q) for _ in range(n)]
    assert [int(x) for x in _ref.negacyclic_mul_schoolbook(a, b, q)] == py_negacyclic(a, b, q)


@pytest.mark.parametrize("n,bits", [(4, 30), (16, 50), (64, 60), (256, 45)])
def test_ntt_product_vs_schoolbook(n, bits):
    q = _ref.gen_primes(int(math.log2(n)), [bits])[0]
    psi = _ref.find_psi(n, q)
    assert pow(psi, n, q) == q - 1
    rng = np.random.default_rng(n)
    a = rng.integers(0, q, n, dtype=np.uint64)
    b = rng.integers(0, q, n, dtype=np.uint64)
    np.testing.assert_array_equal(_ref.negacyclic_mul(a, b, q, psi),
                                  _ref.negacyclic_mul_schoolbook(a, b, q))


def test_monomial_wraparound():
    n, q = 32, _ref.gen_primes(5, [40])[0]
    psi = _ref.find_psi(n, q)
    for i, j in [(0, 5), (7, 30), (31, 31), (16, 16)]:
        a = np.zeros(n, np.uint64)
        b = np.zeros(n, np.uint64)
        a[i] = 1
        b[j] = 1
        c = _ref.negacyclic_mul(a, b, q, psi)
        want = np.zeros(n, np.uint64)
        if i + j < n:
            want[i + j] = 1
        else:
            want[i + j - n] = q - 1
        np.testing.assert_array_equal(c, want)


# ---------------------------------------------------------------- automorphism
@pytest.mark.parametrize("g", [5, 25, 127, 3, 125])
def test_automorphism_is_ring_homomorphism(g):
    n, q = 64, _ref.gen_primes(6, [50])[0]
    psi = _ref.find_psi(n, q)
    rng = np.random.default_rng(g)
    a = rng.integers(0, q, n, dtype=np.uint64)
    b = rng.integers(0, q, n, dtype=np.uint64)
    lhs = _ref.automorphism(_ref.negacyclic_mul(a, b, q, psi), g, q)
    rhs = _ref.negacyclic_mul(_ref.automorphism(a, g, q), _ref.automorphism(b, g, q), q, psi)
    np.testing.assert_array_equal(lhs, rhs)
    # phi_g(phi_h(a)) = phi_{g h}(a), and phi_g(X) = X^g
    h = 5
    np.testing.assert_array_equal(_ref.automorphism(_ref.automorphism(a, h, q), g, q),
                                  _ref.automorphism(a, g * h % (2 * n), q))
    x = np.zeros(n, np.uint64)
    x[1] = 1
    want = np.zeros(n, np.uint64)
    if g % (2 * n) < n:
        want[g % (2 * n)] = 1
    else:
        want[g % (2 * n) - n] = q - 1
    np.testing.assert_array_equal(_ref.automorphism(x, g, q), want)


# ---------------------------------------------------------------- RNS steps
@pytest.mark.parametrize("n_in", [1, 2, 3, 4])
def test_base_convert_is_x_plus_small_multiple(n_in):
    primes = _ref.gen_primes(3, [40] * n_in + [60, 50, 45])
    bp, cp = primes[:n_in], primes[n_in:]
    rng = random.Random(n_in)
    x = rand_res(rng, bp, 8)
    out = _ref.base_convert(x, bp, cp)
    D = 1
    for p in bp:
        D *= p
    for c in range(8):
        X, _ = crt(x[:, c], bp)
        us = [u for u in range(n_in) if all(int(out[k, c]) == (X + u * D) % p
                                             for k, p in enumerate(cp))]
        assert len(us) == 1


@pytest.mark.parametrize("nq,npr", [(2, 1), (3, 2), (5, 4)])
def test_moddown_is_the_centred_conversion(nq, npr):
    """ModDown(u) = (U - C) / P exactly (bigint), C = sum_k y_k (P/p_k) with
    y_k = [u_k (P/p_k)^-1]_{p_k} taken in (-p_k/2, p_k/2]: C = U mod P up to
    a multiple of P, and (U - C)/P - U/P = -sum_k y_k/p_k, centred."""
    primes = _ref.gen_primes(3, [45] * nq + [60] * npr)
    qs, ps = primes[:nq], primes[nq:]
    rng = random.Random(nq * 10 + npr)
    u = rand_res(rng, qs + ps, 8)
    out = _ref.moddown(u, qs, ps)
    P = 1
    for p in ps:
        P *= p
    for c in range(8):
        X, _ = crt(u[:, c], qs + ps)
        C = 0
        for k, p in enumerate(ps):
            hat = P // p
            y = int(u[nq + k, c]) * pow(hat % p, -1, p) % p
            if y > p // 2:
                y -= p
            C += y * hat
        assert (X - C) % P == 0
        want = (X - C) // P
        assert abs(Fraction(X, P) - want) <= Fraction(npr, 2)
        for i, q in enumerate(qs):
            assert int(out[i, c]) == want % q


@pytest.mark.parametrize("nl", [2, 3, 6])
def test_rescale_exact_rounded_division(nl):
    """Rescale by q_l is the nearest integer to X / q_l (q_l odd: no ties)."""
    primes = _ref.gen_primes(3, [60] + [40] * (nl - 1))
    rng = random.Random(nl)
    x = rand_res(rng, primes, 8)
    out = _ref.rescale(x, primes)
    ql = primes[-1]
    for c in range(8):
        X, _ = crt(x[:, c], primes)
        want = (X + (ql - 1) // 2) // ql
        assert abs(Fraction(X, ql) - want) < Fraction(1, 2)
        for i, q in enumerate(primes[:-1]):
            assert int(out[i, c]) == want % q


def test_rescale_error_stays_small_at_low_frequency_slots():
    """The reason rescale rounds: a constant multiplied into a fresh
    ciphertext, then one rescale, at N = 2^15, scale 2^40.  With rounding
    the error is the centred rounding noise e0 + e1 s (4.0e-8 here, about
    4.5 standard deviations of sqrt(N/18) sqrt(N) / 2^40); a floor rescale
    biases every coefficient of both parts by -1/2, and decryption
    multiplies that bias by s and amplifies it at the slots near 1
    (measured: 1.7e-6 with floor)."""
    P = ckks.Params(15, [60] + [40] * 9, [60] * 4, 4, 40)
    s = ckks.keygen_secret(P, 3)
    rng = np.random.default_rng(1)
    z = rng.uniform(-0.05, 0.05, P.slots)
    ct = ckks.encrypt(P, 3, 0, ckks.encode(P, z, P.scale, P.L), s, P.L)
    qL = P.q[P.L]
    acc = np.zeros_like(ct)
    ckks.const_mac(P, acc, ct, int(round(0.06 * qL)))
    r = ckks.rescale_ct(P, acc)
    d = ckks.decode(P, ckks.decrypt(P, r, s), P.scale)
    assert np.max(np.abs(d - 0.06 * z)) < 1e-7


def test_rotation_error_stays_small_at_low_frequency_slots():
    """The reason ModDown's conversion is centred: one rotation at N = 2^15,
    scale 2^40 decrypts within 2e-7 of the rolled slots (7.5e-8 measured);
    the plain conversion biases c1 by -K/2 per coefficient, and decryption
    amplifies that at the slots near 1 (5.2e-6 measured)."""
    P = ckks.Params(15, [60] + [40] * 9, [60] * 4, 4, 40)
    s = ckks.keygen_secret(P, 3)
    rng = np.random.default_rng(1)
    z = rng.uniform(-0.05, 0.05, P.slots)
    ct = ckks.encrypt(P, 3, 0, ckks.encode(P, z, P.scale, P.L), s, P.L)
    r = ckks.rotate(P, ct, 1, ckks.keygen_rotation(P, 3, s, 1))
    d = ckks.decode(P, ckks.decrypt(P, r, s), P.scale)
    assert np.max(np.abs(d - np.roll(z, -1))) < 2e-7


# ---------------------------------------------------------------- encoding
def test_encode_closed_form_n4():
    """N = 4: two slots at zeta^1 and zeta^5, zeta = exp(i pi/4); the encoded
    polynomial evaluated there (by direct evaluation) gives scale * z."""
    P = ckks.Params(2, [20], [20], 1, 10)
    z = np.array([0.75 - 0.25j, -0.5 + 1.0j])
    m = ckks.embed_inverse(P, z)
    zeta = np.exp(1j * np.pi / 4)
    for j, e in enumerate([1, 5]):
        val = sum(m[i] * zeta ** (e * i) for i in range(4))
        assert abs(val - z[j]) < 1e-12
    # conjugate points give the conjugate values (real polynomial)
    for j, e in enumerate([7, 3]):
        val = sum(m[i] * zeta ** (e * i) for i in range(4))
        assert abs(val - np.conj(z[j])) < 1e-12


@pytest.mark.parametrize("log_n", [3, 6, 11])
def test_encode_decode_roundtrip(log_n):
    P = ckks.Params(log_n, [60, 40], [60], 1, 40)
    rng = np.random.default_rng(log_n)
    z = rng.uniform(-2, 2, P.slots)
    pt = ckks.encode(P, z, P.scale, 1)
    zz = ckks.decode(P, pt, P.scale)
    # rounding error: each coefficient moves by <= 1/2, so each slot by <= N/2 / scale
    assert np.max(np.abs(zz - z)) <= P.n / 2 / P.scale
    # direct evaluation of the decoded slots (no FFT) for a few j
    m = [int(v) for v in ckks.crt_centered(P, pt)]
    zeta = np.exp(1j * np.pi / P.n)
    for j in (0, 1, P.slots - 1):
        e = pow(5, j, 2 * P.n)
        val = sum(m[i] * zeta ** (e * i) for i in range(P.n)) / P.scale
        assert abs(val - zz[j]) < 1e-9


def test_round_half_away():
    x = np.array([0.5, -0.5, 1.5, -2.5, 2.0 ** 52 + 1, -(2.0 ** 53) - 2, 0.49999999999999994])
    np.testing.assert_array_equal(ckks.round_half_away(x),
                                  [1, -1, 2, -3, 2.0 ** 52 + 1, -(2.0 ** 53) - 2, 0])


# ---------------------------------------------------------------- encryption
@pytest.fixture(scope="module")
def ctx10():
    P = small_params(log_n=10, nq=4, qb=40, npr=2, alpha=2)
    s = ckks.keygen_secret(P, 5)
    return P, s


def test_samplers_ranges_and_determinism():
    t = _ref.sample_ternary(3, 1, 0, 4096)
    assert set(np.unique(t)) <= {-1, 0, 1} and abs(np.mean(t == 0) - 1 / 3) < 0.05
    e = _ref.sample_gauss(3, 5, 0, 20000)
    assert e.min() >= -19 and e.max() <= 19
    q = _ref.gen_primes(10, [40])
    u = _ref.sample_uniform(3, 4, 0, q, 4096)
    assert u.max() < q[0]
    np.testing.assert_array_equal(u, _ref.sample_uniform(3, 4, 0, q, 4096))
    assert not np.array_equal(u, _ref.sample_uniform(3, 4, 1, q, 4096))
    # SplitMix64 from its published definition (Python ints)
    seed, purpose, index = 12345, 2, 77
    M64 = (1 << 64) - 1

    def mix(z):
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        return z ^ (z >> 31)

    s = mix(seed ^ (purpose << 48) ^ index)
    want = []
    for _ in range(4):
        s = (s + 0x9E3779B97F4A7C15) & M64
        want.append(mix(s))
    assert [int(v) for v in _ref.splitmix(seed, purpose, index, 4)] == want


def test_noise_is_the_discrete_gaussian():
    """The noise sampler against the definition of D_sigma (sigma = 3.2,
    P(x) proportional to exp(-x^2 / (2 sigma^2)), |x| <= 19): frequencies of
    |x| <= 6 within five standard errors of the definition's probabilities,
    the sign symmetric, the variance sigma^2 up to sampling error."""
    n = 400000
    e = np.concatenate([_ref.sample_gauss(7, 5, i, n // 4) for i in range(4)])
    xs = np.arange(-19, 20)
    rho = np.exp(-xs.astype(float) ** 2 / (2 * 3.2 ** 2))
    prob = rho / rho.sum()
    for x in range(-6, 7):
        p = prob[x + 19]
        f = np.mean(e == x)
        assert abs(f - p) < 5 * np.sqrt(p * (1 - p) / n), (x, f, p)
    assert abs(np.mean(e)) < 0.03
    assert abs(np.var(e) - float((prob * xs ** 2).sum())) < 0.15
    assert abs(float((prob * xs ** 2).sum()) - 3.2 ** 2) < 1e-3


def test_encrypt_decrypt_and_add(ctx10):
    P, s = ctx10
    rng = np.random.default_rng(0)
    z1, z2 = rng.uniform(-1, 1, P.slots), rng.uniform(-1, 1, P.slots)
    c1 = ckks.encrypt(P, 5, 0, ckks.encode(P, z1, P.scale, P.L), s, P.L)
    c2 = ckks.encrypt(P, 5, 1, ckks.encode(P, z2, P.scale, P.L), s, P.L)
    d1 = ckks.decrypt(P, c1, s)
    d2 = ckks.decrypt(P, c2, s)
    # Dec(c1 + c2) = Dec(c1) + Dec(c2) exactly on residues (Sec. 2.1)
    np.testing.assert_array_equal(ckks.decrypt(P, ckks.add_ct(P, c1, c2), s),
                                  ckks.add_res(d1, d2, P.q))
    assert np.max(np.abs(ckks.decode(P, d1, P.scale) - z1)) < 2 ** -25
    # the error polynomial is the CBD noise: small and centred
    diff = ckks.crt_centered(P, ckks.sub_res(d1, ckks.encode(P, z1, P.scale, P.L), P.q))
    assert max(abs(int(v)) for v in diff) <= 20


def test_seeded_uniform_sampler_from_the_stream_words():
    """The regenerable uniform sampler against its definition on the pinned
    SplitMix64 stream: coefficient x of limb i is (w_{2k+1} 2^64 + w_{2k})
    mod q_i with k = i n + x and w_j the stream's words (taken here from the
    stream itself, the first 2 n_limbs n of them), for a 40-bit and a
    60-bit prime; every coefficient can be drawn alone, so a different
    index or purpose gives an unrelated sample."""
    q = [int(v) for v in _ref.gen_primes(10, [40, 60])]
    n = 64
    seed, purpose, index = 9, 6, 3
    w = [int(v) for v in _ref.splitmix(seed, purpose, index, 2 * len(q) * n)]
    got = _ref.sample_uniform_wide(seed, purpose, index, q, n)
    for i, qi in enumerate(q):
        for x in range(n):
            k = i * n + x
            assert int(got[i, x]) == ((w[2 * k + 1] << 64) + w[2 * k]) % qi
    assert not np.array_equal(got, _ref.sample_uniform_wide(seed, purpose, index + 1, q, n))


def test_seeded_uniform_sampler_is_uniform():
    """Frequencies of the sampler's values in 16 equal ranges of [0, q)
    within five standard errors of 1/16, and its mean within five standard
    errors of (q - 1)/2, for a 45-bit prime (a dropped high word would leave
    (w_lo mod q), still nearly uniform: the definition test above catches
    that; this one catches a biased or truncated reduction)."""
    q = int(_ref.gen_primes(12, [45])[0])
    u = _ref.sample_uniform_wide(11, 6, 0, [q], 1 << 16)[0].astype(np.float64)
    n = u.size
    counts = np.bincount(np.minimum((u / q * 16).astype(np.int64), 15), minlength=16) / n
    assert np.all(np.abs(counts - 1 / 16) < 5 * np.sqrt((1 / 16) * (15 / 16) / n))
    assert abs(u.mean() - (q - 1) / 2) < 5 * q / np.sqrt(12 * n)


def test_seeded_encryption_decrypts_and_expands_to_a_ciphertext(ctx10):
    """encrypt_seeded: c0 alone, (c0, a) rebuilt from (seed, index); the
    rebuilt ciphertext decrypts to the message plus the Gaussian noise (all
    of it within |e| <= 19, the sampler's tail), and its c1 is the seeded
    uniform sample."""
    P, s = ctx10
    rng = np.random.default_rng(1)
    z = rng.uniform(-1, 1, P.slots)
    pt = ckks.encode(P, z, P.scale, P.L)
    c0 = ckks.encrypt_seeded(P, 5, 2, pt, s, P.L)
    ct = ckks.expand_seeded(P, 5, 2, c0)
    np.testing.assert_array_equal(ct[1], _ref.sample_uniform_wide(5, 6, 2, P.q[:P.L + 1], P.n))
    d = ckks.decrypt(P, ct, s)
    diff = ckks.crt_centered(P, ckks.sub_res(d, pt[:P.L + 1], P.q))
    assert max(abs(int(v)) for v in diff) <= 19
    assert np.max(np.abs(ckks.decode(P, d, P.scale) - z)) < 2 ** -25


def test_pmult_and_rescale(ctx10):
    P, s = ctx10
    rng = np.random.default_rng(1)
    z, w = rng.uniform(-1, 1, P.slots), rng.uniform(-1, 1, P.slots)
    c = ckks.encrypt(P, 5, 2, ckks.encode(P, z, P.scale, P.L), s, P.L)
    ql = P.q[P.L]
    pw = ckks.encode(P, w, float(ql), P.L)
    prod = ckks.pmult(P, pw, c)
    r = ckks.rescale_ct(P, prod)
    assert r.shape[1] == P.L
    got = ckks.decode(P, ckks.decrypt(P, r, s), P.scale)
    assert np.max(np.abs(got - z * w)) < 2 ** -25
    # Dec(rescale(c)) * q_l ~ Dec(c): decode both at matching scales
    before = ckks.decode(P, ckks.decrypt(P, prod, s), P.scale * ql)
    assert np.max(np.abs(before - got)) < 2 ** -25


@pytest.mark.parametrize("alpha,npr", [(1, 1), (2, 2), (3, 3)])
def test_rotation_matches_paper_definition(alpha, npr):
    P = small_params(log_n=10, nq=4, qb=40, npr=npr, alpha=alpha)
    s = ckks.keygen_secret(P, 9)
    rng = np.random.default_rng(alpha)
    z = rng.uniform(-1, 1, P.slots)
    c = ckks.encrypt(P, 9, 0, ckks.encode(P, z, P.scale, P.L), s, P.L)
    for k in (1, -1, 4, -64, 200, P.slots // 2):
        key = ckks.keygen_rotation(P, 9, s, k)
        for lvl_c in (c, ckks.drop_ct(c)):
            got = ckks.decode(P, ckks.decrypt(P, ckks.rotate(P, lvl_c, k, key), s), P.scale)
            want = np.concatenate([z[k % P.slots:], z[:k % P.slots]])
            assert np.max(np.abs(got - want)) < 2 ** -20


def test_rotation_golden_example():
    ex = GOLDEN["rotation_definition"]
    P = ckks.Params(4, [60, 40], [60], 1, 40)     # N = 16: 8 slots
    assert P.slots == ex["slots"]
    s = ckks.keygen_secret(P, 1)
    c = ckks.encrypt(P, 1, 0, ckks.encode(P, np.array(ex["message"], float), P.scale, 1), s, 1)
    got = ckks.decode(P, ckks.decrypt(P, ckks.rotate(P, c, ex["k"], ckks.keygen_rotation(P, 1, s, ex["k"])), s), P.scale)
    np.testing.assert_allclose(got.real, ex["rotated"], atol=1e-6)


def test_internal_sum_golden():
    ex = GOLDEN["internal_sum"]
    P = ckks.Params(4, [60, 40], [60], 1, 40)
    s = ckks.keygen_secret(P, 2)
    c = ckks.encrypt(P, 2, 0, ckks.encode(P, np.array(ex["message"], float), P.scale, 1), s, 1)
    for m in range(ex["rotations"]):
        c = ckks.add_ct(P, c, ckks.rotate(P, c, 1 << m, ckks.keygen_rotation(P, 2, s, 1 << m)))
    got = ckks.decode(P, ckks.decrypt(P, c, s), P.scale)
    np.testing.assert_allclose(got.real, [ex["every_slot"]] * ex["slots"], atol=1e-5)


def test_keyswitch_identity_bigint():
    """After KS, c0' + c1' s = phi_g(c0) + phi_g(c1) phi_g(s) + small (Sec. 2.1
    rotation correctness), checked on CRT-lifted centred integers."""
    P = ckks.Params(5, [60, 40, 40], [60, 60], 2, 40)
    s = ckks.keygen_secret(P, 4)
    rng = random.Random(3)
    c = np.stack([rand_res(rng, P.q, P.n), rand_res(rng, P.q, P.n)])   # arbitrary ciphertext
    k = 3
    g = P.galois(k)
    r = ckks.rotate(P, c, k, ckks.keygen_rotation(P, 4, s, k))
    lhs = ckks.decrypt(P, r, s)
    sg = ckks.automorphism_small(s, g, P.n)
    phi = np.stack([np.stack([_ref.automorphism(c[p, i], g, q) for i, q in enumerate(P.q)]) for p in range(2)])
    rhs = ckks.add_res(phi[0], ckks.poly_mul(P, phi[1], ckks.small_to_res(sg, P.q), P.q), P.q)
    diff = ckks.crt_centered(P, ckks.sub_res(lhs, rhs, P.q))
    assert max(abs(int(v)) for v in diff) < 2 ** 30


# ---------------------------------------------------------------- planner
def test_packing_rule_paper_cases():
    ex = GOLDEN["packing_case_split"]
    for c in ex["t1_cases"]:
        assert planner.choose_t(c["F"], c["n"], c["V"], c["Fp"], c["M"]) == 1
    # J = 2 * (#PMult = #Add = ceil(F n / t)) + cost(Rot) * ceil(log t), Table 1 / App. B.1
    for F, n in [(16, 5), (1433, 4), (7, 3)]:
        for t in (1, 2, 4, 8, 16):
            pm = -(-F * n // t)
            assert planner.packing_objective(t, F, n) == 2 * pm + ex["rot_to_pmult_cost"] * math.ceil(math.log2(t))
    # toy case: J(4) = J(8) = 80 is the minimum, the tie goes to the smaller t
    assert planner.choose_t(16, 5, 64, 8, 2048) == 4


def test_cpoo_merge_golden():
    ex = GOLDEN["cpoo_merge"]
    assert sum(ex["bit_steps"]) == ex["merged"] == ex["shift"]
    # one token of shift 6: radix-2 groups take Rot(2) then Rot(4); a radix-8
    # group covering bits 0..2 takes the single merged Rot(6)
    P = ckks.Params(5, [60] + [40] * 5, [60], 1, 40)
    row_ptr = np.array([0, 1, 1, 1, 1, 1, 1, 1, 1])
    col = np.array([6])      # node 0 aggregates node 6, six slots away
    val = np.array([1.0])
    W = np.ones((1, 1))
    perm = np.arange(8)
    p2 = planner.build_plan(P, P.L, row_ptr, col, val, 8, W, perm, 1, radix_bits=1, aoo=False)
    assert [k for g in p2.groups for (_, k) in g.rotations] == ex["bit_steps"]
    p8 = planner.build_plan(P, P.L, row_ptr, col, val, 8, W, perm, 1, radix_bits=3, aoo=False)
    assert [k for g in p8.groups for (_, k) in g.rotations] == [ex["merged"]]


GRAPHS = [dict(graph="er", V=48, deg=4.0, F=5, Fp=3, seed=1),
          dict(graph="er", V=100, deg=8.0, F=4, Fp=2, seed=2),
          dict(graph="chung_lu", V=200, deg=4.0, gamma=2.2, F=4, Fp=2, x="tfidf", w="glorot", seed=3)]


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
@pytest.mark.parametrize("radix", [1, 2, 4])
@pytest.mark.parametrize("aoo", [True, False])
@pytest.mark.parametrize("order", ["identity", "random"])
def test_plan_simulation_equals_fp64_product(gi, radix, aoo, order):
    """T3: the plan run on plain slot vectors (rotate = np.roll) equals A-hat Z."""
    w = wl.make_workload(**GRAPHS[gi])
    P = ckks.Params(11, [60] + [40] * 14, [60], 1, 40)
    perm = wl.identity_order(w.V) if order == "identity" else wl.random_order(w.V, P.slots, gi)
    plan = planner.build_plan(P, P.L, w.row_ptr, w.col, w.val, w.V, w.W, perm, 1, radix, aoo)
    Z = planner.simulate_combination(plan, w.X, w.W)
    ref = w.reference_output()
    for j in range(plan.Fp):
        np.testing.assert_allclose(Z[j][perm], (w.X @ w.W)[:, j], atol=1e-12)
        out = planner.simulate_aggregation(plan, Z[j])
        assert np.max(np.abs(out[perm] - ref[:, j])) < 1e-12
        mask = np.ones(plan.M, bool)
        mask[perm] = False
        assert np.all(out[mask] == 0)
    # one source slot feeds one output slot per lane: masks of one (src, k) into one lane
    # never overlap with each other (each (src, k, dst) is a single term)
    for g in plan.groups:
        keys = [(tm.src, tm.k, tm.dst) for tm in g.terms]
        assert len(keys) == len(set(keys))


@pytest.mark.parametrize("t", [2, 4])
def test_plan_simulation_packed_t(t):
    w = wl.make_workload(graph="er", V=40, deg=3.0, F=7, Fp=3, seed=5)
    P = ckks.Params(10, [60] + [40] * 12, [60], 1, 40)
    perm = wl.random_order(w.V, P.slots // t, 4)
    plan = planner.build_plan(P, P.L, w.row_ptr, w.col, w.val, w.V, w.W, perm, t, 2)
    assert plan.comb_rots == [(P.slots // t) << i for i in range(int(math.log2(t)))]
    Z = planner.simulate_combination(plan, w.X, w.W)
    ref = w.reference_output()
    for j in range(plan.Fp):
        out = planner.simulate_aggregation(plan, Z[j])
        assert np.max(np.abs(out[perm] - ref[:, j])) < 1e-12


@pytest.mark.parametrize("seed", range(4))
def test_worst_case_rotation_bound(seed):
    """Sec. 3.3.1: at most (n-1) log^2 rotations per ciphertext, nodes in
    consecutive slots, radix 2."""
    w = wl.make_workload(graph="er", V=64 + 32 * seed, deg=3.0 + seed, F=2, Fp=1, seed=seed)
    P = ckks.Params(11, [60] + [40] * 14, [60], 1, 40)
    plan = planner.build_plan(P, P.L, w.row_ptr, w.col, w.val, w.V, w.W,
                              wl.identity_order(w.V), 1, 1, aoo=False)
    n = w.max_degree()
    bound = (n - 1) * math.ceil(math.log2(w.V)) ** 2
    assert sum(len(g.rotations) for g in plan.groups) <= bound


# ---------------------------------------------------------------- end to end
def test_layer_decrypts_to_fp64_product():
    """T2 on a small layer: decrypted output within 2^-20 of A-hat X W."""
    P = ckks.Params(10, [60] + [40] * 6, [60, 60], 2, 40)
    w = wl.make_workload(graph="er", V=24, deg=3.0, F=6, Fp=2, seed=8)
    perm = wl.random_order(w.V, P.slots, 8)
    plan = planner.build_plan(P, P.L, w.row_ptr, w.col, w.val, w.V, w.W, perm, 1, 3)
    s = ckks.keygen_secret(P, 8)
    keys = {k: ckks.keygen_rotation(P, 8, s, k) for k in plan.rotation_amounts()}
    cts = []
    for f in range(w.X.shape[1]):
        v = np.zeros(P.slots)
        v[perm] = w.X[:, f]
        cts.append(ckks.encrypt(P, 8, f, ckks.encode(P, v, P.scale, P.L), s, P.L))
    pts = layer.encode_plan_masks(P, plan)
    outs = layer.layer_axw(P, plan, cts, keys, pts)
    ref = w.reference_output()
    for j, o in enumerate(outs):
        assert o.shape[1] - 1 == plan.out_level
        d = ckks.decode(P, ckks.decrypt(P, o, s), P.scale).real
        assert np.max(np.abs(d[perm] - ref[:, j])) < 2 ** -20


# ---------------------------------------------------------------- planted slips
def test_planted_mistakes_are_caught(monkeypatch):
    """Slips planted in the oracle (on the CPU) fail the pins above."""
    # 1. automorphism without the sign flip breaks the homomorphism pin
    def no_sign(a, g, q):
        a = np.asarray(a, np.uint64)
        n = a.size
        out = np.zeros_like(a)
        for i in range(n):
            out[(i * g) % (2 * n) % n] = a[i]
        return out
    monkeypatch.setattr(_ref, "automorphism", no_sign)
    with pytest.raises(AssertionError):
        test_automorphism_is_ring_homomorphism(5)
    monkeypatch.undo()
    # 2. wrong rotation direction in the planner breaks T3
    monkeypatch.setattr(planner, "shift_amount",
                        lambda s, d, M, aoo=True: (d - s) % M if not aoo else ((d - s) % M if (d - s) % M <= M // 2 else (d - s) % M - M))
    with pytest.raises(AssertionError):
        test_plan_simulation_equals_fp64_product(0, 2, True, "random")
    monkeypatch.undo()
    # 3. a transposed weight use breaks the combination against X W
    orig = planner.simulate_combination

    def transposed(plan, X, W):
        return orig(plan, X, np.ascontiguousarray(W[::-1]))
    monkeypatch.setattr(planner, "simulate_combination", transposed)
    with pytest.raises(AssertionError):
        test_plan_simulation_equals_fp64_product(0, 1, False, "identity")


@pytest.mark.parametrize("nq,npr", [(2, 1), (4, 3)])
def test_moddown_of_p_multiple_is_exact(nq, npr):
    """ModDown(A + P*B) = ModDown(A) + B exactly (B given on the q-limbs, zero
    on the special primes): the identity that lets masked rotations and kept
    values of one output share a single ModDown."""
    primes = _ref.gen_primes(4, [45] * nq + [60] * npr)
    qs, ps = primes[:nq], primes[nq:]
    rng = random.Random(nq)
    A = rand_res(rng, qs + ps, 16)
    B = rand_res(rng, qs, 16)
    P = 1
    for p in ps:
        P *= p
    APB = A.copy()
    for i, q in enumerate(qs):
        APB[i] = ckks.add_res(A[i:i + 1], _ref.mul_scalar(B[i], P % q, q)[None], [q])[0]
    lhs = _ref.moddown(APB, qs, ps)
    rhs = ckks.add_res(_ref.moddown(A, qs, ps), B, qs)
    np.testing.assert_array_equal(lhs, rhs)


# ---------------------------------------------------------------- CMult (x^2)
def test_secret_square_is_the_integer_negacyclic_square():
    P = ckks.Params(10, [60, 40], [60], 1, 40)
    s = ckks.keygen_secret(P, 4).astype(np.int64)
    full = np.convolve(s, s)                      # integer product, then X^N = -1
    want = full[:P.n].copy()
    want[:P.n - 1] -= full[P.n:]
    np.testing.assert_array_equal(ckks.secret_square(P, ckks.keygen_secret(P, 4)), want)


def test_tensor_product_decrypts_to_the_product_bigint():
    """d0 + d1 s + d2 s^2 == (a0 + a1 s)(b0 + b1 s) mod Q, checked on CRT-lifted
    big integers with schoolbook products (N = 16)."""
    P = ckks.Params(4, [50, 40, 40], [60], 1, 30)
    rng = np.random.default_rng(2)
    s = ckks.keygen_secret(P, 2)
    a = np.stack([np.stack([rng.integers(0, q, P.n, dtype=np.uint64) for q in P.q]) for _ in range(2)])
    b = np.stack([np.stack([rng.integers(0, q, P.n, dtype=np.uint64) for q in P.q]) for _ in range(2)])
    d0, d1, d2 = ckks.mul_ct(P, a, b)
    Q = 1
    for q in P.q:
        Q *= q

    def lift(res):
        return [int(v) for v in ckks.crt_centered(P, res)]

    def nmul(x, y):
        out = [0] * P.n
        for i in range(P.n):
            for j in range(P.n):
                k = i + j
                if k < P.n:
                    out[k] += x[i] * y[j]
                else:
                    out[k - P.n] -= x[i] * y[j]
        return out

    si = [int(v) for v in s]
    s2 = nmul(si, si)
    lhs = [x + y + z for x, y, z in zip(lift(d0), nmul(lift(d1), si), nmul(lift(d2), s2))]
    da = [x + y for x, y in zip(lift(a[0]), nmul(lift(a[1]), si))]
    db = [x + y for x, y in zip(lift(b[0]), nmul(lift(b[1]), si))]
    rhs = nmul(da, db)
    assert all((x - y) % Q == 0 for x, y in zip(lhs, rhs))


def test_relinearisation_keeps_the_decryption_up_to_small_noise():
    """Dec(relinearize(d)) - (d0 + d1 s + d2 s^2) is the key-switching noise:
    small against the scale (bigint check at N = 1024)."""
    P = ckks.Params(10, [60, 40, 40, 40], [60, 60], 2, 40)
    s = ckks.keygen_secret(P, 6)
    key = ckks.keygen_relin(P, 6, s)
    rng = np.random.default_rng(3)
    lvl = 3
    z = rng.uniform(-1, 1, P.slots)
    ct = ckks.encrypt(P, 6, 0, ckks.encode(P, z, P.scale, lvl), s, lvl)
    d0, d1, d2 = ckks.mul_ct(P, ct, ct)
    r = ckks.relinearize(P, d0, d1, d2, key)
    s_res = ckks.small_to_res(s, P.q[:lvl + 1])
    s2_res = ckks.small_to_res(ckks.secret_square(P, s), P.q[:lvl + 1])
    qs = P.q[:lvl + 1]
    want = ckks.add_res(ckks.add_res(d0, ckks.poly_mul(P, d1, s_res, qs), qs),
                        ckks.poly_mul(P, d2, s2_res, qs), qs)
    got = ckks.decrypt(P, r, s)
    diff = [abs(int(v)) for v in ckks.crt_centered(P, ckks.sub_res(got, want, qs))]
    assert max(diff) < 2 ** 30 and max(diff) > 0


def test_cmult_decodes_to_the_product():
    P = ckks.Params(11, [60, 40, 40, 40], [60, 60], 2, 40)
    s = ckks.keygen_secret(P, 8)
    key = ckks.keygen_relin(P, 8, s)
    rng = np.random.default_rng(4)
    z1, z2 = rng.uniform(-1, 1, P.slots), rng.uniform(-1, 1, P.slots)
    lvl = 3
    c1 = ckks.encrypt(P, 8, 0, ckks.encode(P, z1, P.scale, lvl), s, lvl)
    c2 = ckks.encrypt(P, 8, 1, ckks.encode(P, z2, P.scale, lvl), s, lvl)
    out = ckks.mul_relin_rescale(P, c1, c2, key)
    assert out.shape[1] == lvl
    d = ckks.decode(P, ckks.decrypt(P, out, s), P.scale * P.scale / P.q[lvl])
    assert np.max(np.abs(d - z1 * z2)) < 2 ** -20


def test_planted_cmult_mistakes_are_caught(monkeypatch):
    """A dropped cross term in the tensor product, and s in place of s^2 in
    the relinearisation key, each fail a CMult pin."""
    orig = ckks.mul_ct

    def dropped(params, a, b):
        d0, d1, d2 = orig(params, a, b)
        primes = params.q[:a.shape[1]]
        return d0, ckks.poly_mul(params, a[0], b[1], primes), d2
    monkeypatch.setattr(ckks, "mul_ct", dropped)
    with pytest.raises(AssertionError):
        test_tensor_product_decrypts_to_the_product_bigint()
    monkeypatch.undo()
    monkeypatch.setattr(ckks, "secret_square", lambda params, s: np.asarray(s, np.int64))
    with pytest.raises(AssertionError):
        test_cmult_decodes_to_the_product()


# ------------------------------------------------ learned planner's latency model
def _mlp_case(seed=0, n=40, n_in=5, h=7):
    from oracle import mlp
    rng = np.random.default_rng(seed)
    params = [rng.normal(0, 0.5, s) for s in mlp.sizes(n_in, h)]
    X = rng.normal(0, 1, (n, n_in))
    y = rng.normal(0, 1, n)
    return mlp, params, X, y


def test_mlp_gradient_matches_finite_differences():
    mlp, params, X, y = _mlp_case()
    loss, grads = mlp.loss_and_grads(params, X, y)
    flat = mlp.pack(params)
    g = mlp.pack(grads)
    eps = 1e-6
    for i in range(flat.size):
        up, dn = flat.copy(), flat.copy()
        up[i] += eps
        dn[i] -= eps
        lu, _ = mlp.loss_and_grads(mlp.unpack(up, 5, 7), X, y)
        ld, _ = mlp.loss_and_grads(mlp.unpack(dn, 5, 7), X, y)
        assert abs((lu - ld) / (2 * eps) - g[i]) < 1e-6 * max(1.0, abs(g[i]))


def test_mlp_adam_fits_a_linear_target():
    """With a linear target the network can fit exactly; full-batch Adam
    drives the error far below the target's variance."""
    from oracle import mlp
    rng = np.random.default_rng(1)
    X = rng.uniform(0, 1, (200, 4))
    y = X @ np.array([1.0, -2.0, 0.5, 3.0]) + 0.25
    params = [rng.normal(0, 0.3, s) for s in mlp.sizes(4, 16)]
    _, losses = mlp.adam(params, X, y, 1500, 0.01)
    assert losses[-1] < 1e-3 * np.var(y) and losses[-1] < losses[0]


def test_planted_mlp_mistake_is_caught(monkeypatch):
    """A transposed weight in the backward pass fails the finite-difference
    pin."""
    from oracle import mlp
    orig = mlp.loss_and_grads

    def transposed(params, X, y):
        loss, g = orig(params, X, y)
        W1, b1, W2, b2, W3, b3 = params
        f, (z1, a1, z2, a2) = mlp.forward(params, X)
        n = X.shape[0]
        d3 = (2.0 / n) * (f - y)[:, None]
        d2 = (d3 @ W3.T) * (z2 > 0)
        d1 = (d2 @ W2) * (z1 > 0)          # W2 instead of W2^T
        g[0] = X.T @ d1
        g[1] = d1.sum(axis=0)
        return loss, g
    monkeypatch.setattr(mlp, "loss_and_grads", transposed)
    with pytest.raises(AssertionError):
        test_mlp_gradient_matches_finite_differences()
