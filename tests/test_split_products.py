"""The word-level bounds the CUDA kernels' unreduced sums of products rely
on, emulated on the host in 64-bit wrapping arithmetic (numpy uint64) and
checked against exact integer sums.

Split products: a factor below 2^46 is split into 23-bit halves
v = v0 + v1 2^23, and a sum of T products is kept as three 64-bit partial
sums A0 = sum v0 m0, A1 = sum (v0 m1 + v1 m0), A2 = sum v1 m1.  Karatsuba's
form keeps K = sum (v0 + v1)(m0 + m1) instead of A1 and recovers
A1 = K - A0 - A2.  Both must give S = A0 + A1 2^23 + A2 2^46 exactly, for up
to 2^16 terms, with S below q 2^64 (Montgomery's condition)."""
import numpy as np
import pytest

M23 = np.uint64((1 << 23) - 1)


def split(v):
    return v & M23, v >> np.uint64(23)


def sums(v, m):
    """Column sums in uint64 (wrapping), as the kernels keep them."""
    v0, v1 = split(v)
    m0, m1 = split(m)
    with np.errstate(over="ignore"):
        a0 = np.sum(v0 * m0, dtype=np.uint64)
        a1 = np.sum(v0 * m1 + v1 * m0, dtype=np.uint64)
        a2 = np.sum(v1 * m1, dtype=np.uint64)
        k = np.sum((v0 + v1) * (m0 + m1), dtype=np.uint64)
        a1k = k - a0 - a2
    return int(a0), int(a1), int(a2), int(a1k)


@pytest.mark.parametrize("T", [1, 2, 255, 1 << 16])
@pytest.mark.parametrize("kind", ["random", "max"])
def test_split_and_karatsuba_sums_are_exact(T, kind):
    q = (1 << 46) - 27          # a word bound: every factor is below 2^46
    rng = np.random.default_rng(T)
    if kind == "max":
        v = np.full(T, q - 1, np.uint64)
        m = np.full(T, q - 1, np.uint64)
    else:
        v = rng.integers(0, q, T, dtype=np.uint64)
        m = rng.integers(0, q, T, dtype=np.uint64)
    a0, a1, a2, a1k = sums(v, m)
    exact = sum(int(x) * int(y) for x, y in zip(v, m))
    assert a1k == a1                                    # Karatsuba's middle sum is the same integer
    assert a0 + (a1 << 23) + (a2 << 46) == exact        # no partial sum wrapped
    assert exact < q << 64                              # Montgomery's condition


def test_karatsuba_factor_and_product_bounds():
    """Half sums below 2^24, their products below 2^48: 2^16 of them below 2^64."""
    h = (1 << 23) - 1
    assert 2 * h < 1 << 24
    assert (2 * h) ** 2 < 1 << 48
    assert (1 << 16) * (2 * h) ** 2 < 1 << 64


M30 = np.uint64((1 << 30) - 1)


def split30_sums(v, m):
    v0, v1 = v & M30, v >> np.uint64(30)
    m0, m1 = m & M30, m >> np.uint64(30)
    with np.errstate(over="ignore"):
        a0 = np.sum(v0 * m0, dtype=np.uint64)
        a1 = np.sum(v0 * m1 + v1 * m0, dtype=np.uint64)
        a2 = np.sum(v1 * m1, dtype=np.uint64)
    return int(a0), int(a1), int(a2)


@pytest.mark.parametrize("T", [1, 8])
def test_thirty_bit_sums_hold_eight_terms_of_sixty_bit_words(T):
    """Factors below 2^60 in 30-bit halves: the three partial sums of up to
    eight products (the key switch's digits, the group MAC's fold period on
    the 60-bit primes) do not wrap, so the 128-bit total is exact."""
    w = np.full(T, (1 << 60) - 1, np.uint64)
    a0, a1, a2 = split30_sums(w, w)
    assert a0 + (a1 << 30) + (a2 << 60) == T * ((1 << 60) - 1) ** 2


def test_montgomery_condition_for_the_group_mac_and_key_switch_sums():
    """The unreduced sums stay below q 2^64, the condition of one Montgomery
    reduction: 255 products of reduced factors (a group-MAC output per
    launch) for q < 2^46, and up to 8 products of factors below 2^60 for a
    60-bit q (the key switch's split path)."""
    q46 = (1 << 46) - 1
    assert 255 * q46 * q46 < q46 << 64
    q60 = (1 << 60) - 1
    assert 8 * ((1 << 60) - 1) * q60 < q60 << 64
