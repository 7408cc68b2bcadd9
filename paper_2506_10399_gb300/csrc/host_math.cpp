// host_math.cpp -- host-side number theory, seeded sampling and the FP64
// CKKS encoder of the library.
#include <cmath>
#include <complex>
#include <cstring>

#include "fg_internal.h"

namespace hm {

u64 mulmod(u64 a, u64 b, u64 q) { return (u64)((u128)a * b % q); }

u64 powmod(u64 a, u64 e, u64 q)
{
    u64 r = 1 % q;
    a %= q;
    for (; e; e >>= 1) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
    }
    return r;
}

u64 invmod(u64 a, u64 q) { return powmod(a, q - 2, q); }   // q prime

// Miller-Rabin, witnesses = first 12 primes: exact for all 64-bit integers
bool is_prime(u64 n)
{
    static const u64 w[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 p : w) {
        if (n == p) return true;
        if (n % p == 0) return false;
    }
    u64 d = n - 1;
    int s = 0;
    while (!(d & 1)) d >>= 1, s++;
    for (u64 a : w) {
        u64 x = powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s && comp; r++) {
            x = mulmod(x, x, n);
            if (x == n - 1) comp = false;
        }
        if (comp) return false;
    }
    return true;
}

std::vector<u64> gen_primes(int log_n, const std::vector<int> &bits)
{
    const u64 step = 2ull << log_n;   // primes must be 1 mod 2N
    std::vector<u64> out;
    for (int b : bits) {
        FG_CHECK(b >= log_n + 2 && b <= 60, FG_EINVAL, "prime bit size out of range");
        u64 c = (1ull << b) - step + 1;
        bool found = false;
        for (; c > step; c -= step) {
            bool used = false;
            for (u64 p : out) used |= (p == c);
            if (!used && is_prime(c)) {
                out.push_back(c);
                found = true;
                break;
            }
        }
        FG_CHECK(found, FG_EINVAL, "no NTT-friendly prime of the requested size");
    }
    return out;
}

// a primitive 2N-th root of unity: psi = x^((q-1)/2N) with psi^N = -1
u64 find_psi(int n, u64 q)
{
    u64 e = (q - 1) / (2 * (u64)n);
    for (u64 x = 2; x < q; x++) {
        u64 psi = powmod(x, e, q);
        if (powmod(psi, n, q) == q - 1) return psi;
    }
    throw fg_error(FG_EINVAL, "no 2N-th root of unity");
}

u64 shoup(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

u64 mont_qneg(u64 q)
{
    u64 inv = q;                       // Newton: each step doubles the correct bits
    for (int i = 0; i < 6; i++) inv *= 2 - q * inv;
    return (u64)0 - inv;
}

u64 to_mont(u64 x, u64 q) { return (u64)(((u128)(x % q) << 64) % q); }

int bitrev(int x, int bits)
{
    int r = 0;
    for (int i = 0; i < bits; i++) r = (r << 1) | ((x >> i) & 1);
    return r;
}

// ------------------------------------------------------------------ SplitMix64
static inline u64 sm_mix(u64 z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

Stream::Stream(u64 seed, u64 purpose, u64 index) : s(sm_mix(seed ^ (purpose << 48) ^ index)) {}

u64 Stream::next()
{
    s += 0x9E3779B97F4A7C15ull;
    return sm_mix(s);
}

void sample_ternary(u64 seed, u64 purpose, u64 index, int n, int8_t *out)
{
    Stream st(seed, purpose, index);
    for (int i = 0; i < n; i++) {
        u64 r;
        do r = st.next() >> 62; while (r == 3);
        out[i] = (int8_t)((int)r - 1);
    }
}

// Noise: the discrete Gaussian D_sigma, sigma = 3.2 (P(x) proportional to
// exp(-x^2 / (2 sigma^2))), cut at |x| <= 19 (6 sigma).  Inversion of a
// cumulative table over |x|: T[k] = floor(2^63 sum_{i<=k} p_i / S), p_0 =
// rho(0), p_i = 2 rho(i) for i >= 1 (both signs; zero counted once), S the
// sum of all p_i, T[19] = 2^63.  One stream word r per coefficient: |x| =
// the least k with (r >> 1) < T[k], negative when bit 0 of r is set.
static void gauss_table(u64 *T)
{
    const int tail = 19;
    const double sigma = 3.2, two_s2 = 2.0 * sigma * sigma;
    double p[20], S = 0.0, c = 0.0;
    for (int k = 0; k <= tail; k++) {
        const double r = std::exp(-(double)(k * k) / two_s2);
        p[k] = k == 0 ? r : 2.0 * r;
        S += p[k];
    }
    for (int k = 0; k < tail; k++) {
        c += p[k];
        T[k] = (u64)(c / S * 9223372036854775808.0);
    }
    T[tail] = 1ull << 63;
}

void sample_gauss(u64 seed, u64 purpose, u64 index, int n, int8_t *out)
{
    u64 T[20];
    gauss_table(T);
    Stream st(seed, purpose, index);
    for (int i = 0; i < n; i++) {
        const u64 r = st.next(), u = r >> 1;
        int k = 0;
        while (u >= T[k]) k++;
        out[i] = (int8_t)((r & 1) && k ? -k : k);
    }
}

// Coefficient x of limb l from the stream's words 2(l n + x) and
// 2(l n + x) + 1 (word j of a SplitMix64 stream is mix(s0 + (j + 1) gamma)),
// (w_hi 2^64 + w_lo) mod q_l: every coefficient can be drawn on its own.
void sample_uniform_wide(u64 seed, u64 purpose, u64 index, const u64 *primes, int n_limbs, int n,
                         u64 *out)
{
    const u64 s0 = Stream(seed, purpose, index).s, gamma = 0x9E3779B97F4A7C15ull;
    for (int l = 0; l < n_limbs; l++) {
        const u64 q = primes[l];
        for (int x = 0; x < n; x++) {
            const u64 j = 2 * ((u64)l * (u64)n + (u64)x);
            const u64 lo = sm_mix(s0 + (j + 1) * gamma), hi = sm_mix(s0 + (j + 2) * gamma);
            const unsigned __int128 w = ((unsigned __int128)hi << 64) | lo;
            out[(size_t)l * n + x] = (u64)(w % q);
        }
    }
}

void sample_uniform(u64 seed, u64 purpose, u64 index, const u64 *primes, int n_limbs, int n,
                    u64 *out)
{
    Stream st(seed, purpose, index);
    for (int l = 0; l < n_limbs; l++) {
        u64 q = primes[l];
        int bl = 64 - __builtin_clzll(q);
        u64 mask = bl == 64 ? ~0ull : ((1ull << bl) - 1);
        u64 *o = out + (size_t)l * n;
        for (int i = 0; i < n; i++) {
            u64 r;
            do r = st.next() & mask; while (r >= q);
            o[i] = r;
        }
    }
}

// ------------------------------------------------------------------ encoder
double round_half_away(double x) { return std::round(x); }

typedef std::complex<double> cd;

// in-place radix-2 DFT, sign = -1: X_k = sum x_j e^{-2 pi i jk/n}; sign = +1 the other way
static void fft(std::vector<cd> &a, int sign)
{
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; i++) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        const double ang = sign * 2.0 * M_PI / (double)len;
        std::vector<cd> w(len / 2);
        for (size_t k = 0; k < len / 2; k++) w[k] = cd(std::cos(ang * k), std::sin(ang * k));
        for (size_t i = 0; i < n; i += len)
            for (size_t k = 0; k < len / 2; k++) {
                cd u = a[i + k], v = a[i + k + len / 2] * w[k];
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
    }
}

// slot j <-> evaluation at zeta^(5^j mod 2N), zeta = exp(i pi / N); the
// conjugate slot sits at 2N - 5^j.  Coefficients: m_i = (1/N) sum over the
// 2N-th roots e of m(zeta^e) zeta^(-e i), a length-2N DFT.
void encode(int log_n, const double *slots, int n_slots, double scale, const u64 *primes,
            int n_limbs, u64 *out)
{
    const int n = 1 << log_n, m = n / 2, two_n = 2 * n;
    FG_CHECK(n_slots >= 0 && n_slots <= m, FG_EINVAL, "too many slot values");
    std::vector<cd> v(two_n, cd(0, 0));
    u64 e = 1;
    for (int j = 0; j < m; j++) {
        double z = j < n_slots ? slots[j] : 0.0;
        FG_CHECK(std::isfinite(z), FG_EINVAL, "slot value is not finite");
        v[e] = cd(z, 0);
        v[two_n - e] = cd(z, 0);
        e = e * 5 % two_n;
    }
    fft(v, -1);
    for (int i = 0; i < n; i++) {
        double c = round_half_away(scale * v[i].real() / n);
        FG_CHECK(std::fabs(c) < 9.2e18, FG_EINVAL, "encoded coefficient overflows 63 bits");
        i64 ci = (i64)c;
        for (int l = 0; l < n_limbs; l++) {
            i64 q = (i64)primes[l];
            i64 r = ci % q;
            out[(size_t)l * n + i] = (u64)(r < 0 ? r + q : r);
        }
    }
}

void decode(int log_n, const double *coef, double *slots_out)
{
    const int n = 1 << log_n, m = n / 2, two_n = 2 * n;
    std::vector<cd> u(two_n, cd(0, 0));
    for (int i = 0; i < n; i++) u[i] = cd(coef[i], 0);
    fft(u, +1);    // u[e] = sum_i m_i zeta^(e i)
    u64 e = 1;
    for (int j = 0; j < m; j++) {
        slots_out[j] = u[e].real();
        e = e * 5 % two_n;
    }
}

}  // namespace hm
