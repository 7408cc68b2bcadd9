/*
 * ckks_ref.c -- reference CKKS-RNS arithmetic, TEST INFRASTRUCTURE ONLY.
 *
 * This is the oracle's exact-integer core: plain, slow and meant to be read
 * against the definitions.  Nothing in the library links or calls it; only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark load
 * it (through ctypes, see _ref.py).
 *
 * Conventions
 *   - A polynomial over a list of primes is stored limb-major:
 *     u64[n_limbs][N], every residue canonical in [0, q).
 *   - All products are exact: (unsigned __int128)a*b % q.
 *   - Negacyclic means the ring Z_q[X]/(X^N + 1) of the CKKS preliminaries
 *     (paper, Sec. 2.1: R_Q = Z_Q[X]/(X^N+1), Q = prod q_i).
 *
 * Parity status of each function is stated beside it; the pins live in
 * tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* scalar modular arithmetic                                           */
/* ------------------------------------------------------------------ */

static u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static u64 addmod(u64 a, u64 b, u64 q) { u64 s = a + b; return s >= q ? s - q : s; }
static u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + (q - b); }

static u64 powmod(u64 b, u64 e, u64 q)
{
    u64 r = 1 % q;
    b %= q;
    while (e) {
        if (e & 1) r = mulmod(r, b, q);
        b = mulmod(b, b, q);
        e >>= 1;
    }
    return r;
}

/* inverse modulo a prime, by Fermat's little theorem */
static u64 invmod(u64 a, u64 q) { return powmod(a % q, q - 2, q); }

u64 ref_mulmod(u64 a, u64 b, u64 q) { return mulmod(a, b, q); }
u64 ref_powmod(u64 a, u64 e, u64 q) { return powmod(a, e, q); }
u64 ref_invmod(u64 a, u64 q) { return invmod(a, q); }

/* ------------------------------------------------------------------ */
/* primes                                                              */
/* ------------------------------------------------------------------ */

/* Miller-Rabin with the first twelve primes as witnesses; this set is
 * deterministic for every n < 3.3e24, hence for every 64-bit n. */
int ref_is_prime(u64 n)
{
    static const u64 wit[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == wit[i]) return 1;
        if (n % wit[i] == 0) return 0;
    }
    u64 d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        u64 x = powmod(wit[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int comp = 1;
        for (int r = 1; r < s; r++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { comp = 0; break; }
        }
        if (comp) return 0;
    }
    return 1;
}

/* For each requested bit size b (in order) take the largest prime q < 2^b
 * with q = 1 (mod 2N) that was not taken before.  q = 1 (mod 2N) is what
 * makes a primitive 2N-th root of unity exist mod q, so the negacyclic
 * product can go through an NTT.  Returns 0, or -1 if a size runs dry. */
int ref_gen_primes(int log_n, int count, const int *bits, u64 *out)
{
    u64 two_n = 2ull << log_n;
    for (int i = 0; i < count; i++) {
        if (bits[i] < log_n + 2 || bits[i] > 62) return -1;
        u64 top = 1ull << bits[i];
        u64 c = top - two_n + 1; /* largest value < 2^b that is 1 mod 2N */
        int found = 0;
        while (c > two_n) {
            int used = 0;
            for (int j = 0; j < i; j++) if (out[j] == c) used = 1;
            if (!used && ref_is_prime(c)) { out[i] = c; found = 1; break; }
            c -= two_n;
        }
        if (!found) return -1;
    }
    return 0;
}

/* A primitive 2N-th root of unity mod q: x^((q-1)/2N) for the smallest
 * x >= 2 whose power psi has psi^N = -1 (then psi has order exactly 2N). */
u64 ref_find_psi(int n, u64 q)
{
    u64 e = (q - 1) / (2 * (u64)n);
    for (u64 x = 2; x < q; x++) {
        u64 psi = powmod(x, e, q);
        if (powmod(psi, (u64)n, q) == q - 1) return psi;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* negacyclic products                                                 */
/* ------------------------------------------------------------------ */

/* The definition: c = a*b in Z_q[X]/(X^N+1), i.e. X^N = -1.  O(N^2). */
void ref_negacyclic_mul_schoolbook(const u64 *a, const u64 *b, u64 *c, int n, u64 q)
{
    for (int k = 0; k < n; k++) c[k] = 0;
    for (int i = 0; i < n; i++) {
        for (int j = 0; j < n; j++) {
            u64 p = mulmod(a[i], b[j], q);
            int k = i + j;
            if (k < n) c[k] = addmod(c[k], p, q);
            else c[k - n] = submod(c[k - n], p, q);
        }
    }
}

static unsigned bitrev(unsigned x, int bits)
{
    unsigned r = 0;
    for (int i = 0; i < bits; i++) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

/* Textbook iterative radix-2 DFT over Z_q: X_k = sum_j x_j w^(jk), with w a
 * primitive n-th root of unity (bit-reversal permutation, then log n rounds
 * of butterflies).  In place. */
static void cyclic_dft(u64 *x, int n, u64 w, u64 q)
{
    int logn = 0;
    while ((1 << logn) < n) logn++;
    for (int i = 0; i < n; i++) {
        int j = (int)bitrev((unsigned)i, logn);
        if (j > i) { u64 t = x[i]; x[i] = x[j]; x[j] = t; }
    }
    for (int len = 2; len <= n; len <<= 1) {
        u64 wl = powmod(w, (u64)(n / len), q); /* primitive len-th root */
        for (int i = 0; i < n; i += len) {
            u64 wj = 1;
            for (int j = 0; j < len / 2; j++) {
                u64 u = x[i + j];
                u64 v = mulmod(x[i + j + len / 2], wj, q);
                x[i + j] = addmod(u, v, q);
                x[i + j + len / 2] = submod(u, v, q);
                wj = mulmod(wj, wl, q);
            }
        }
    }
}

/* Negacyclic product through the convolution theorem: with psi a primitive
 * 2N-th root, a(X)b(X) mod X^N+1 equals psi^-i * cyclic_conv(psi^i a, psi^i b),
 * and the cyclic convolution is DFT^-1(DFT(.) . DFT(.)) with w = psi^2. */
void ref_negacyclic_mul(const u64 *a, const u64 *b, u64 *c, int n, u64 q, u64 psi)
{
    u64 *ta = (u64 *)malloc(sizeof(u64) * (size_t)n);
    u64 *tb = (u64 *)malloc(sizeof(u64) * (size_t)n);
    u64 w = mulmod(psi, psi, q);
    u64 pw = 1;
    for (int i = 0; i < n; i++) {
        ta[i] = mulmod(a[i], pw, q);
        tb[i] = mulmod(b[i], pw, q);
        pw = mulmod(pw, psi, q);
    }
    cyclic_dft(ta, n, w, q);
    cyclic_dft(tb, n, w, q);
    for (int i = 0; i < n; i++) ta[i] = mulmod(ta[i], tb[i], q);
    cyclic_dft(ta, n, invmod(w, q), q); /* inverse DFT up to the factor 1/n */
    u64 ninv = invmod((u64)n, q);
    u64 psi_inv = invmod(psi, q);
    pw = ninv;
    for (int i = 0; i < n; i++) {
        c[i] = mulmod(ta[i], pw, q);
        pw = mulmod(pw, psi_inv, q);
    }
    free(ta);
    free(tb);
}

/* ------------------------------------------------------------------ */
/* automorphism X -> X^g (rotation, Sec. 2.1)                          */
/* ------------------------------------------------------------------ */

/* out(X) = a(X^g) mod X^N+1 for odd g: coefficient i moves to i*g mod 2N,
 * with a sign flip when that exponent lands in [N, 2N). */
void ref_automorphism(const u64 *a, u64 *out, int n, u64 g, u64 q)
{
    u64 two_n = 2 * (u64)n;
    for (int i = 0; i < n; i++) {
        u64 e = ((u64)i * g) % two_n;
        if (e < (u64)n) out[e] = a[i];
        else out[e - n] = a[i] ? q - a[i] : 0;
    }
}

/* ------------------------------------------------------------------ */
/* approximate fast base conversion                                    */
/* ------------------------------------------------------------------ */

/* Conv_{B -> C}(x)_p = sum_i [x_i * (B/b_i)^-1]_{b_i} * (B/b_i)  mod p,
 * for every target prime p of C, with no correction of the overflow term
 * (the result equals x + u*B for some 0 <= u < n_in).  Used by ModUp
 * (B = one key-switching digit) and by ModDown (B = P).
 * in: u64[n_in][n], out: u64[n_out][n]. */
void ref_base_convert(const u64 *in, int n_in, const u64 *b_primes,
                      u64 *out, int n_out, const u64 *c_primes, int n)
{
    /* (B/b_i)^-1 mod b_i, and (B/b_i) mod p for each target p */
    u64 *hat_inv = (u64 *)malloc(sizeof(u64) * (size_t)n_in);
    u64 *hat_mod = (u64 *)malloc(sizeof(u64) * (size_t)n_in * (size_t)n_out);
    for (int i = 0; i < n_in; i++) {
        u64 bi = b_primes[i];
        u64 h = 1;
        for (int j = 0; j < n_in; j++) if (j != i) h = mulmod(h, b_primes[j] % bi, bi);
        hat_inv[i] = invmod(h, bi);
        for (int k = 0; k < n_out; k++) {
            u64 p = c_primes[k];
            u64 hp = 1;
            for (int j = 0; j < n_in; j++) if (j != i) hp = mulmod(hp, b_primes[j] % p, p);
            hat_mod[(size_t)i * n_out + k] = hp;
        }
    }
    for (int x = 0; x < n; x++) {
        for (int k = 0; k < n_out; k++) out[(size_t)k * n + x] = 0;
        for (int i = 0; i < n_in; i++) {
            u64 y = mulmod(in[(size_t)i * n + x], hat_inv[i], b_primes[i]);
            for (int k = 0; k < n_out; k++) {
                u64 p = c_primes[k];
                u64 t = mulmod(y % p, hat_mod[(size_t)i * n_out + k], p);
                out[(size_t)k * n + x] = addmod(out[(size_t)k * n + x], t, p);
            }
        }
    }
    free(hat_inv);
    free(hat_mod);
}

/* ------------------------------------------------------------------ */
/* rescale and ModDown                                                 */
/* ------------------------------------------------------------------ */

/* Rescale by the last prime (the level drop that follows a product),
 * rounding to the nearest integer: c <- floor((c + h) / q_l) with
 * h = (q_l - 1) / 2, i.e. per limb
 *   c_i <- (c_i + [h]_{q_i} - [r]_{q_i}) * q_l^-1 mod q_i,  r = [c_l + h]_{q_l}
 * (r in [0, q_l) taken as an integer).  Rounding keeps the error of each
 * coefficient centred; a floor (h = 0) biases every coefficient of both
 * parts by -1/2, and that constant bias, multiplied by s at decryption,
 * is amplified at the slots whose evaluation points lie near 1.
 * in: [l+1][n] over q_0..q_l, out: [l][n]. */
void ref_rescale(const u64 *in, int n_limbs, const u64 *primes, u64 *out, int n)
{
    int l = n_limbs - 1;
    u64 ql = primes[l];
    u64 h = (ql - 1) / 2;
    const u64 *c = in + (size_t)l * n;
    for (int i = 0; i < l; i++) {
        u64 qi = primes[i];
        u64 inv = invmod(ql % qi, qi);
        u64 hi = h % qi;
        for (int x = 0; x < n; x++) {
            u64 r = addmod(c[x], h, ql);
            u64 d = submod(addmod(in[(size_t)i * n + x], hi, qi), r % qi, qi);
            out[(size_t)i * n + x] = mulmod(d, inv, qi);
        }
    }
}

/* ModDown with the centred fast base conversion: with
 *   y_k = [u_k (P/p_k)^-1]_{p_k} taken in (-p_k/2, p_k/2],
 *   Conv'(u)_i = sum_k y_k (P/p_k) mod q_i   (= [u]_P + e P, |e| <= K/2),
 * out_i = (u_i - Conv'(u)_i) * P^-1 mod q_i.  As integers out = (u - Conv')/P,
 * whose distance to u/P is minus S = sum_k y_k / p_k: centred, so the error
 * has mean zero (the plain conversion, y_k in [0, p_k), gives mean -K/2,
 * and that constant bias in c1 is amplified at decryption at the slots near
 * 1).  Conv' is the plain conversion minus c P, c = #{k : y_k > p_k/2}.
 * in: [nq + np][n] with the q-limbs first, out: [nq][n]. */
void ref_moddown(const u64 *in, int nq, const u64 *q_primes, int np,
                 const u64 *p_primes, u64 *out, int n)
{
    u64 *conv = (u64 *)malloc(sizeof(u64) * (size_t)nq * (size_t)n);
    int *c = (int *)calloc((size_t)n, sizeof(int));
    ref_base_convert(in + (size_t)nq * n, np, p_primes, conv, nq, q_primes, n);
    for (int k = 0; k < np; k++) {
        u64 pk = p_primes[k], h = 1;
        for (int j = 0; j < np; j++) if (j != k) h = mulmod(h, p_primes[j] % pk, pk);
        u64 hinv = invmod(h, pk);
        for (int x = 0; x < n; x++)
            if (mulmod(in[(size_t)(nq + k) * n + x], hinv, pk) > pk / 2) c[x]++;
    }
    for (int i = 0; i < nq; i++) {
        u64 qi = q_primes[i];
        u64 P = 1;
        for (int k = 0; k < np; k++) P = mulmod(P, p_primes[k] % qi, qi);
        u64 pinv = invmod(P, qi);
        for (int x = 0; x < n; x++) {
            u64 cv = submod(conv[(size_t)i * n + x], mulmod((u64)c[x], P, qi), qi);
            u64 d = submod(in[(size_t)i * n + x], cv, qi);
            out[(size_t)i * n + x] = mulmod(d, pinv, qi);
        }
    }
    free(c);
    free(conv);
}

/* ------------------------------------------------------------------ */
/* limb-wise helpers                                                   */
/* ------------------------------------------------------------------ */

void ref_mul_scalar(const u64 *a, u64 s, u64 *out, int n, u64 q)
{
    for (int x = 0; x < n; x++) out[x] = mulmod(a[x], s, q);
}

/* out += a * s  (mod q) */
void ref_mac_scalar(const u64 *a, u64 s, u64 *out, int n, u64 q)
{
    for (int x = 0; x < n; x++) out[x] = addmod(out[x], mulmod(a[x], s, q), q);
}

/* ------------------------------------------------------------------ */
/* seeded sampling                                                     */
/* ------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15, then the output
 * mix z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27; z *= 0x94D049BB133111EB;
 * z ^= z>>31.  A stream (seed, purpose, index) starts from the state
 * mix(seed ^ (purpose << 48) ^ index).  Not a cryptographic generator. */
static u64 sm_mix(u64 z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

typedef struct { u64 s; } sm_stream;

static sm_stream sm_open(u64 seed, u64 purpose, u64 index)
{
    sm_stream st;
    st.s = sm_mix(seed ^ (purpose << 48) ^ index);
    return st;
}

static u64 sm_next(sm_stream *st)
{
    st->s += 0x9E3779B97F4A7C15ull;
    return sm_mix(st->s);
}

u64 ref_splitmix_first(u64 seed, u64 purpose, u64 index, int count, u64 *out)
{
    sm_stream st = sm_open(seed, purpose, index);
    for (int i = 0; i < count; i++) out[i] = sm_next(&st);
    return count ? out[0] : 0;
}

/* ternary secret: per coefficient draw r = next >> 62 until r < 3, value r-1 */
void ref_sample_ternary(u64 seed, u64 purpose, u64 index, int n, i64 *out)
{
    sm_stream st = sm_open(seed, purpose, index);
    for (int x = 0; x < n; x++) {
        u64 r;
        do { r = sm_next(&st) >> 62; } while (r == 3);
        out[x] = (i64)r - 1;
    }
}

/* noise: the discrete Gaussian D_sigma on the integers, sigma = 3.2, i.e.
 * P(x) proportional to rho(x) = exp(-x^2 / (2 sigma^2)), cut at |x| <= 19
 * (6 sigma), sampled by inversion of a cumulative distribution table over
 * |x|: T[k] = floor(2^63 * sum_{i <= k} p_i / S) with p_0 = rho(0), p_i =
 * 2 rho(i) (both signs) for i >= 1 and S = sum of all p_i (so zero is not
 * counted twice), T[19] = 2^63.  One draw r per coefficient: |x| = the
 * least k with (r >> 1) < T[k], and x = -|x| when bit 0 of r is set. */
#define REF_GAUSS_TAIL 19

void ref_gauss_table(u64 *T)
{
    const double sigma = 3.2, two_s2 = 2.0 * sigma * sigma;
    double p[REF_GAUSS_TAIL + 1], S = 0.0, c = 0.0;
    for (int k = 0; k <= REF_GAUSS_TAIL; k++) {
        const double r = exp(-(double)(k * k) / two_s2);
        p[k] = k == 0 ? r : 2.0 * r;
        S += p[k];
    }
    for (int k = 0; k < REF_GAUSS_TAIL; k++) {
        c += p[k];
        T[k] = (u64)(c / S * 9223372036854775808.0);
    }
    T[REF_GAUSS_TAIL] = 1ull << 63;
}

void ref_sample_gauss(u64 seed, u64 purpose, u64 index, int n, i64 *out)
{
    u64 T[REF_GAUSS_TAIL + 1];
    ref_gauss_table(T);
    sm_stream st = sm_open(seed, purpose, index);
    for (int x = 0; x < n; x++) {
        u64 r = sm_next(&st);
        u64 u = r >> 1;
        int k = 0;
        while (u >= T[k]) k++;
        out[x] = (r & 1) && k ? -(i64)k : (i64)k;
    }
}

/* uniform residues from two stream words each, without rejection, so that
 * every coefficient can be drawn on its own: coefficient x of limb i takes
 * the stream's words number 2(i n + x) and 2(i n + x) + 1 (counted from 0),
 * w_lo and w_hi, and is (w_hi 2^64 + w_lo) mod q_i (a bias below
 * q_i / 2^128).  The word number j of a SplitMix64 stream is
 * mix(s0 + (j + 1) * 0x9E3779B97F4A7C15) with s0 the stream's start state.
 * out: u64[n_limbs][n]. */
void ref_sample_uniform_wide(u64 seed, u64 purpose, u64 index, const u64 *primes,
                             int n_limbs, int n, u64 *out)
{
    const u64 s0 = sm_open(seed, purpose, index).s;
    for (int i = 0; i < n_limbs; i++) {
        const u64 q = primes[i];
        for (int x = 0; x < n; x++) {
            const u64 j = 2 * ((u64)i * (u64)n + (u64)x);
            const u64 lo = sm_mix(s0 + (j + 1) * 0x9E3779B97F4A7C15ull);
            const u64 hi = sm_mix(s0 + (j + 2) * 0x9E3779B97F4A7C15ull);
            const unsigned __int128 w = ((unsigned __int128)hi << 64) | lo;
            out[(size_t)i * n + x] = (u64)(w % q);
        }
    }
}

/* uniform residues: limb by limb in the order given, coefficient by
 * coefficient, draw r = next & (2^bitlen(q) - 1) until r < q.
 * out: u64[n_limbs][n]. */
void ref_sample_uniform(u64 seed, u64 purpose, u64 index, const u64 *primes,
                        int n_limbs, int n, u64 *out)
{
    sm_stream st = sm_open(seed, purpose, index);
    for (int i = 0; i < n_limbs; i++) {
        u64 q = primes[i];
        int bl = 64 - __builtin_clzll(q);
        u64 mask = bl == 64 ? ~0ull : ((1ull << bl) - 1);
        for (int x = 0; x < n; x++) {
            u64 r;
            do { r = sm_next(&st) & mask; } while (r >= q);
            out[(size_t)i * n + x] = r;
        }
    }
}
