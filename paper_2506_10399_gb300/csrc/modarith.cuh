// modarith.cuh -- 64-bit modular arithmetic on CUDA cores for RNS-CKKS.
//
// All primes are below 2^62, so lazy values in [0, 4q) fit a 64-bit word.
// Methods (each a published one):
//   * Shoup's precomputed-quotient multiplication by a fixed operand w
//     (w' = floor(w 2^64 / q)), lazy form in [0, 2q) as in Harvey, "Faster
//     arithmetic for number-theoretic transforms" (J. Symb. Comp. 2014).
//   * Montgomery reduction (Montgomery, Math. Comp. 1985) with R = 2^64 for
//     products of two variable operands, one operand kept in Montgomery form.
#pragma once
#include <cstdint>

typedef uint64_t u64;
typedef uint32_t u32;

// per-prime constants kept on the device
struct PrimeC {
    u64 q;       // the prime
    u64 qneg;    // -q^-1 mod 2^64 (Montgomery)
    u64 r2;      // R^2 mod q, R = 2^64 (to enter Montgomery form)
    u64 one_s;   // floor(2^64 / q): Shoup companion of 1 (full reduction of a word)
};

__device__ __forceinline__ u64 mulhi64(u64 a, u64 b) { return __umul64hi(a, b); }

// a * w mod q in [0, 2q), any a < 2^64 (Harvey's lazy Shoup product)
__device__ __forceinline__ u64 shoup_lazy(u64 a, u64 w, u64 ws, u64 q)
{
    return a * w - mulhi64(a, ws) * q;
}

__device__ __forceinline__ u64 reduce2(u64 x, u64 q) { return x >= q ? x - q : x; }

__device__ __forceinline__ u64 reduce4(u64 x, u64 q)
{
    x = x >= 2 * q ? x - 2 * q : x;
    return x >= q ? x - q : x;
}

// a * w mod q in [0, q)
__device__ __forceinline__ u64 shoup_mul(u64 a, u64 w, u64 ws, u64 q)
{
    return reduce2(shoup_lazy(a, w, ws, q), q);
}

// x mod q for any 64-bit x
__device__ __forceinline__ u64 reduce_word(u64 x, const PrimeC &P)
{
    return shoup_mul(x, 1, P.one_s, P.q);
}

// Montgomery reduction of T = hi 2^64 + lo < q 2^64: T R^-1 mod q in [0, q).
// With m = lo * (-q^-1) mod 2^64, lo + (m q mod 2^64) is 0 when lo == 0 and
// exactly 2^64 otherwise, so the carry into the high word is (lo != 0).
__device__ __forceinline__ u64 redc(u64 hi, u64 lo, const PrimeC &P)
{
    u64 m = lo * P.qneg;
    u64 t = hi + mulhi64(m, P.q) + (lo != 0);
    return reduce2(t, P.q);
}

// a * b R^-1 mod q (one of a, b in Montgomery form gives the plain product)
__device__ __forceinline__ u64 mont_mul(u64 a, u64 b, const PrimeC &P)
{
    return redc(mulhi64(a, b), a * b, P);
}

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) { return reduce2(a + b, q); }
__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

// 128-bit accumulator: (hi, lo) += a * b
__device__ __forceinline__ void mac128(u64 &hi, u64 &lo, u64 a, u64 b)
{
    u64 p_lo = a * b;
    u64 p_hi = mulhi64(a, b);
    lo += p_lo;
    hi += p_hi + (lo < p_lo);
}
