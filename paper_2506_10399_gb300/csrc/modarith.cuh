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
// (one carry-chained multiply-add pair, so no compare is needed for the carry)
__device__ __forceinline__ void mac128(u64 &hi, u64 &lo, u64 a, u64 b)
{
    asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\t"
        "madc.hi.u64 %1, %2, %3, %1;"
        : "+l"(lo), "+l"(hi)
        : "l"(a), "l"(b));
}

// Products of factors below 2^46 on 32-bit multipliers.  A factor is
// stored split into 23-bit halves, v0 | v1 << 32 (v = v0 + v1 2^23), and a
// sum of products is kept as three 64-bit partial sums
//   A0 = sum v0 m0,  A1 = sum (v0 m1 + v1 m0),  A2 = sum v1 m1,
// each term below 2^47, so up to 2^16 terms cannot overflow.  Four
// 32 x 32 -> 64-bit multiply-adds per product replace the 64 x 64 -> 128-bit
// product of mac128.
__device__ __forceinline__ u64 split23(u64 v) { return (v & 0x7FFFFF) | ((v >> 23) << 32); }

__device__ __forceinline__ void mac_split(u64 &a0, u64 &a1, u64 &a2, u64 v, u64 m)
{
    const u32 v0 = (u32)v, v1 = (u32)(v >> 32), m0 = (u32)m, m1 = (u32)(m >> 32);
    asm("mad.wide.u32 %0, %3, %5, %0;\n\t"
        "mad.wide.u32 %1, %3, %6, %1;\n\t"
        "mad.wide.u32 %1, %4, %5, %1;\n\t"
        "mad.wide.u32 %2, %4, %6, %2;"
        : "+l"(a0), "+l"(a1), "+l"(a2)
        : "r"(v0), "r"(v1), "r"(m0), "r"(m1));
}

// (A0 + A1 2^23 + A2 2^46) R^-1 mod q.  The sum S = A0 + A1 2^23 + A2 2^46
// of T < 2^16 products of reduced factors is below T q^2, so its high word
// is below T q (q / 2^64) < q / 4 for q < 2^46: Montgomery's condition
// S < q 2^64 holds without reducing the high word first.
__device__ __forceinline__ u64 fold_split(u64 a0, u64 a1, u64 a2, const PrimeC &P)
{
    u64 lo = a0, hi = (a1 >> 41) + (a2 >> 18);
    u64 t = a1 << 23;
    lo += t;
    hi += lo < t;
    t = a2 << 46;
    lo += t;
    hi += lo < t;
    return redc(hi, lo, P);
}



// Factors below 2^60 split into 30-bit halves, v0 | v1 << 32 (v = v0 + v1
// 2^30): the same three partial sums, each product below 2^60, so they hold
// 8 terms (A1 takes two products a term) before they are folded into a
// 128-bit total.
__device__ __forceinline__ u64 split30(u64 v) { return (v & 0x3FFFFFFF) | ((v >> 30) << 32); }

// (hi, lo) += A0 + A1 2^30 + A2 2^60
__device__ __forceinline__ void fold30(u64 &hi, u64 &lo, u64 a0, u64 a1, u64 a2)
{
    lo += a0;
    hi += lo < a0;
    u64 t = a1 << 30;
    lo += t;
    hi += (lo < t) + (a1 >> 34);
    t = a2 << 60;
    lo += t;
    hi += (lo < t) + (a2 >> 4);
}

// Shoup product with a three-product quotient that skips the carries of the
// low partial products: h = y_hi w'_hi + hi(y_lo w'_hi) + hi(y_hi w'_lo)
// leaves out y_lo w'_lo and the low halves of the cross products, three
// terms below 2^64 each, so h is floor(y w' / 2^64) or up to two less and
// y w - h q lies in [0, 4q) for any y < 2^64 (q < 2^61).
__device__ __forceinline__ u64 shoup_lazy4(u64 y, u64 w, u64 ws, u64 q)
{
    const u32 y0 = (u32)y, y1 = (u32)(y >> 32);
    const u32 s0 = (u32)ws, s1 = (u32)(ws >> 32);
    const u64 c = (u64)__umulhi(y0, s1) + __umulhi(y1, s0);
    u64 h;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(h) : "r"(y1), "r"(s1), "l"(c));
    return y * w - h * q;
}
