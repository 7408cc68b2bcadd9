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
// 32 x 32 -> 64-bit products per product of factors replace the
// 64 x 64 -> 128-bit product of mac128.  Each is added to its partial sum,
// kept as two 32-bit words, by a carry-chained pair: the low word of the
// product into the low word (carry out), the high word of the product plus
// that carry into the high word.  (The same sums as 64-bit mad.wide.u32
// accumulation; measured on GB300, the pairs free registers and issue
// slots: key switch 66.8 -> 59.0 ms, group MAC 87.2 -> 84.5 ms per layer.)
__device__ __forceinline__ u64 split23(u64 v) { return (v & 0x7FFFFF) | ((v >> 23) << 32); }

__device__ __forceinline__ void mac_split(u64 &a0, u64 &a1, u64 &a2, u64 v, u64 m)
{
    const u32 v0 = (u32)v, v1 = (u32)(v >> 32), m0 = (u32)m, m1 = (u32)(m >> 32);
    asm("{\n\t.reg .u32 l0, h0, l1, h1, l2, h2;\n\t"
        "mov.b64 {l0, h0}, %0;\n\tmov.b64 {l1, h1}, %1;\n\tmov.b64 {l2, h2}, %2;\n\t"
        "mad.lo.cc.u32 l0, %3, %5, l0;\n\tmadc.hi.u32 h0, %3, %5, h0;\n\t"
        "mad.lo.cc.u32 l1, %3, %6, l1;\n\tmadc.hi.u32 h1, %3, %6, h1;\n\t"
        "mad.lo.cc.u32 l1, %4, %5, l1;\n\tmadc.hi.u32 h1, %4, %5, h1;\n\t"
        "mad.lo.cc.u32 l2, %4, %6, l2;\n\tmadc.hi.u32 h2, %4, %6, h2;\n\t"
        "mov.b64 %0, {l0, h0};\n\tmov.b64 %1, {l1, h1};\n\tmov.b64 %2, {l2, h2};\n\t}"
        : "+l"(a0), "+l"(a1), "+l"(a2)
        : "r"(v0), "r"(v1), "r"(m0), "r"(m1));
}

// Karatsuba's form of mac_split (Karatsuba and Ofman, 1962): the middle
// partial sum is kept as K = sum (v0 + v1)(m0 + m1) (half sums below 2^24,
// products below 2^48, so again up to 2^16 terms fit), and
// A1 = K - A0 - A2, the same integer as mac_split's A1, is recovered once,
// at the fold (fold_kara): three products and two 32-bit adds per product
// of factors.  Factors below 2^46 only.
__device__ __forceinline__ void mac_kara(u64 &a0, u64 &k, u64 &a2, u64 v, u64 m)
{
    const u32 v0 = (u32)v, v1 = (u32)(v >> 32), m0 = (u32)m, m1 = (u32)(m >> 32);
    const u32 vs = v0 + v1, ms = m0 + m1;
    asm("{\n\t.reg .u32 l0, h0, l1, h1, l2, h2;\n\t"
        "mov.b64 {l0, h0}, %0;\n\tmov.b64 {l1, h1}, %1;\n\tmov.b64 {l2, h2}, %2;\n\t"
        "mad.lo.cc.u32 l0, %3, %5, l0;\n\tmadc.hi.u32 h0, %3, %5, h0;\n\t"
        "mad.lo.cc.u32 l1, %7, %8, l1;\n\tmadc.hi.u32 h1, %7, %8, h1;\n\t"
        "mad.lo.cc.u32 l2, %4, %6, l2;\n\tmadc.hi.u32 h2, %4, %6, h2;\n\t"
        "mov.b64 %0, {l0, h0};\n\tmov.b64 %1, {l1, h1};\n\tmov.b64 %2, {l2, h2};\n\t}"
        : "+l"(a0), "+l"(k), "+l"(a2)
        : "r"(v0), "r"(v1), "r"(m0), "r"(m1), "r"(vs), "r"(ms));
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

__device__ __forceinline__ u64 fold_kara(u64 a0, u64 k, u64 a2, const PrimeC &P)
{
    return fold_split(a0, k - a0 - a2, a2, P);
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
