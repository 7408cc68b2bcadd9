// kernels.cu -- sm_103a kernels of the encrypted GCN layer.
//
// Every kernel works on 64-bit RNS words with the reductions of
// modarith.cuh on CUDA cores.  Layouts are limb-major: a polynomial limb is
// N consecutive words; a batch of limbs is addressed as rows of `per_row`
// limbs (row r, column c at base + (r * row_stride + c) * N), and limb
// column c is reduced modulo prime pidx[c] (pidx < 0: leave that limb).
#include <cstdio>

#include "fg_internal.h"
#include "modarith.cuh"

namespace {

constexpr int kPidxMax = 1024;

struct Batch {
    u64 *src;          // read from
    u64 *dst;          // written to (may equal src)
    int src_stride;    // limbs between rows
    int dst_stride;
    int per_row;
    int rows;
    int8_t pidx[kPidxMax];
};

Batch make_batch(u64 *src, int src_stride, u64 *dst, int dst_stride, int per_row, int rows,
                 const std::vector<int> &pidx)
{
    FG_CHECK(per_row <= kPidxMax && (int)pidx.size() == per_row, FG_EINVAL,
             "limb batch wider than the prime-index table");
    Batch b;
    b.src = src;
    b.dst = dst;
    b.src_stride = src_stride;
    b.dst_stride = dst_stride;
    b.per_row = per_row;
    b.rows = rows;
    for (int i = 0; i < per_row; i++) b.pidx[i] = (int8_t)pidx[i];
    return b;
}

fg_ctx *g_launch_ctx = nullptr;   // context of the wrapper being run (for launch counting)

inline void check_launch(const char *what, int kernels = 1)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw fg_error(FG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    if (g_launch_ctx) g_launch_ctx->launches += kernels;
}

// ------------------------------------------------------------------------
// NTT: negacyclic, Cooley-Tukey forward with twiddles psi^brv(m+i) (natural
// order in, bit-reversed order out: out[j] = a(psi^(2 brv(j) + 1))),
// Gentleman-Sande inverse, Harvey's lazy butterflies.  N = N1 * N2 with
// N1 = 2^s1: pass A runs stages 0..s1-1 on the N2 stride-N2 columns, pass B
// runs the remaining stages inside each of the N1 contiguous rows.
// ------------------------------------------------------------------------
constexpr int kNttThreads = 256;
constexpr int kColsA = 16;       // columns per CTA in pass A
constexpr int kElemsB = 2048;    // elements per CTA in pass B

__device__ __forceinline__ void ct_bfly(u64 &X, u64 &Y, const ulonglong2 w, u64 q, u64 q2)
{
    X = X >= q2 ? X - q2 : X;               // X < 2q, Y < 4q in; both < 4q out
    const u64 T = shoup_lazy(Y, w.x, w.y, q);
    Y = X - T + q2;
    X = X + T;
}

__device__ __forceinline__ void gs_bfly(u64 &X, u64 &Y, const ulonglong2 w, u64 q, u64 q2)
{
    const u64 U = X, V = Y;                 // both < 2q in and out
    const u64 S = U + V;
    X = S >= q2 ? S - q2 : S;
    Y = shoup_lazy(U - V + q2, w.x, w.y, q);
}

// ------------------------------------------------------------------------
// log N = 16: radix-16 rounds.  Every thread holds 16 elements in registers
// for four stages, so each pass makes two shared-memory round trips
// (N = 256 x 256; pass A on columns, pass B on rows).  For primes below
// 2^47 the butterflies skip every conditional reduction and use the
// three-product quotient without carries (shoup_lazy4, products in
// [0, 4q)): forward values grow by at most 4q per stage (< 65q after 16
// stages); inverse values are below 2^(k+1) q after k stages (< 2^64 for
// q < 2^47); one reduction at the end restores [0, q).  Larger primes keep
// Harvey's bounds (< 4q, < 2q).
// ------------------------------------------------------------------------
// tw(st, g): twiddle of group g at stage st (0..3) of the 16-point round
template <bool LAZY, class TW>
__device__ __forceinline__ void ct16(u64 (&v)[16], TW tw, u64 q, u64 q2)
{
#pragma unroll
    for (int st = 0; st < 4; st++) {
        const int h = 8 >> st;
#pragma unroll
        for (int m = 0; m < 16; m++) {
            if ((m & h) == 0) {
                const ulonglong2 w = tw(st, m >> (4 - st));
                u64 X = v[m], Y = v[m + h];
                if (LAZY) {
                    const u64 T = shoup_lazy4(Y, w.x, w.y, q);
                    v[m + h] = X - T + 4 * q;
                    v[m] = X + T;
                } else {
                    X = X >= q2 ? X - q2 : X;
                    const u64 T = shoup_lazy(Y, w.x, w.y, q);
                    v[m + h] = X - T + q2;
                    v[m] = X + T;
                }
            }
        }
    }
}

// k0: number of inverse stages already applied to these values (lazy bound 2^k0 q)
template <bool LAZY, class TW>
__device__ __forceinline__ void gs16(u64 (&v)[16], TW tw, u64 q, u64 q2, int k0)
{
#pragma unroll
    for (int st = 3; st >= 0; st--) {
        const int h = 8 >> st;
        const u64 qb = LAZY ? (q << (k0 + 4 - st)) : q2;   // above the bound of V
#pragma unroll
        for (int m = 0; m < 16; m++) {
            if ((m & h) == 0) {
                const ulonglong2 w = tw(st, m >> (4 - st));
                const u64 U = v[m], V = v[m + h];
                const u64 S = U + V;
                v[m] = LAZY ? S : (S >= q2 ? S - q2 : S);
                v[m + h] = LAZY ? shoup_lazy4(U - V + qb, w.x, w.y, q)
                                : shoup_lazy(U - V + qb, w.x, w.y, q);
            }
        }
    }
}

// A round's 15 twiddles either held in registers for the whole round
// (OD = false: loaded up front) or loaded where each stage uses them (OD =
// true: fewer live registers, so more CTAs per SM).
template <bool OD, class F>
struct Twiddles {
    ulonglong2 w[OD ? 1 : 15];
    F f;
    __device__ __forceinline__ explicit Twiddles(F g) : f(g)
    {
        if (!OD) {
#pragma unroll
            for (int st = 0; st < 4; st++)
#pragma unroll
                for (int gg = 0; gg < (1 << st); gg++) w[OD ? 0 : (1 << st) - 1 + gg] = f(st, gg);
        }
    }
    __device__ __forceinline__ ulonglong2 operator()(int st, int g) const
    {
        return OD ? f(st, g) : w[OD ? 0 : (1 << st) - 1 + g];
    }
};
template <bool OD, class F>
__device__ __forceinline__ Twiddles<OD, F> twiddles(F f) { return Twiddles<OD, F>(f); }

constexpr int kR16Row = 272;   // 256 elements + 16 pad words per row (pass B shared memory)
__device__ __forceinline__ int pad16(int pos) { return pos + (pos >> 4); }

// Tiles: pass A takes COLS (16 or 8) of the 256 columns per CTA, one
// thread per (column, group of 16 rows), 16 x COLS threads; pass B takes
// ROWS (16 or 8) of the 256 rows per CTA, 16 threads per row.  Both tile
// sizes compute the same transform word for word; the batched form picks
// one per shape by timing.
// pass A's two rounds on values already in registers (element (r + 16 m) of
// this thread's column), written to d (the tile's first column)
template <bool LAZY, int COLS, bool OD>
__device__ __forceinline__ void fwd_a16_rounds(u64 (&v)[16], u64 *d, const ulonglong2 *stw, u64 q, u64 *sm)
{
    const int t = threadIdx.x, c = t % COLS, r = t / COLS;   // r: r0 in round 1, r1 in round 2
    constexpr int N2 = 256;
    const u64 q2 = 2 * q;
    // stage st, group g at (1 << st) + g
    ct16<LAZY>(v, twiddles<OD>([&](int st, int g) { return stw[(1 << st) + g]; }), q, q2);
#pragma unroll
    for (int m = 0; m < 16; m++) sm[(r + 16 * m) * COLS + c] = v[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 16; m++) v[m] = sm[(16 * r + m) * COLS + c];
    ct16<LAZY>(v, twiddles<OD>([&](int st, int g) { return stw[(1 << (st + 4)) + (r << st) + g]; }), q, q2);
#pragma unroll
    for (int m = 0; m < 16; m++) d[(size_t)(16 * r + m) * N2 + c] = v[m];   // lazy
}

template <bool LAZY, int COLS, bool OD>
__device__ __forceinline__ void fwd_a16_body(const u64 *s, u64 *d, const ulonglong2 *stw, u64 q, u64 *sm)
{
    const int t = threadIdx.x, c = t % COLS, r = t / COLS;
    constexpr int N2 = 256;
    u64 v[16];
#pragma unroll
    for (int m = 0; m < 16; m++) v[m] = s[(size_t)(r + 16 * m) * N2 + c];
    fwd_a16_rounds<LAZY, COLS, OD>(v, d, stw, q, sm);
}

template <int COLS, bool OD>
__global__ void __launch_bounds__(16 * COLS, (OD ? 64 : 48) / COLS)
ntt16_fwd_a(const Batch bt, const PrimeC *__restrict__ primes, const ulonglong2 *__restrict__ tw)
{
    const int limb = blockIdx.y;
    const int col = limb % bt.per_row, row = limb / bt.per_row;
    const int pi = bt.pidx[col];
    if (pi < 0) return;
    __shared__ u64 sm[256 * COLS];
    __shared__ ulonglong2 stw[256];
    const u64 q = primes[pi].q;
    const ulonglong2 *twp = tw + (size_t)pi * 65536;
    for (int k = threadIdx.x; k < 256; k += blockDim.x) stw[k] = twp[k];
    __syncthreads();
    const int c0 = blockIdx.x * COLS;
    const u64 *src = bt.src + ((size_t)row * bt.src_stride + col) * 65536 + c0;
    u64 *dst = bt.dst + ((size_t)row * bt.dst_stride + col) * 65536 + c0;
    if (q < (1ull << 47)) fwd_a16_body<true, COLS, OD>(src, dst, stw, q, sm);
    else fwd_a16_body<false, COLS, OD>(src, dst, stw, q, sm);
}

template <bool LAZY, bool OD>
__device__ __forceinline__ void fwd_b16_body(u64 *d, const ulonglong2 *twp, const ulonglong2 *rows,
                                             int row0, const PrimeC &P, u64 *sm)
{
    const int t = threadIdx.x, j = t & 15, r = t >> 4;
    constexpr int S1 = 8;
    const u64 q = P.q, q2 = 2 * q;
    u64 v[16];
    const int grow = row0 + r;
    u64 *drow = d + (size_t)r * 256;
#pragma unroll
    for (int m = 0; m < 16; m++) v[m] = drow[j + 16 * m];
    ct16<LAZY>(v, twiddles<OD>([&](int st, int g) { return twp[(1 << (S1 + st)) + (grow << st) + g]; }), q, q2);
    u64 *srow = sm + r * kR16Row;
#pragma unroll
    for (int m = 0; m < 16; m++) srow[pad16(j + 16 * m)] = v[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 16; m++) v[m] = srow[pad16(16 * j + m)];
    // row stages 12..15 from the row-blocked table (consecutive per row)
    ct16<LAZY>(v, twiddles<OD>([&](int st, int g) { return rows[((size_t)grow * 15 + (1 << st) - 1 + g) * 16 + j]; }),
               q, q2);
    ulonglong2 *o = reinterpret_cast<ulonglong2 *>(drow + 16 * j);
#pragma unroll
    for (int m = 0; m < 16; m += 2)
        o[m / 2] = LAZY ? make_ulonglong2(reduce_word(v[m], P), reduce_word(v[m + 1], P))
                        : make_ulonglong2(reduce4(v[m], q), reduce4(v[m + 1], q));
}

template <int ROWS, bool OD>
__global__ void __launch_bounds__(16 * ROWS, (OD ? 64 : 48) / ROWS)
ntt16_fwd_b(const Batch bt, const PrimeC *__restrict__ primes, const ulonglong2 *__restrict__ tw,
            const ulonglong2 *__restrict__ tw_rows)
{
    const int limb = blockIdx.y;
    const int col = limb % bt.per_row, row = limb / bt.per_row;
    const int pi = bt.pidx[col];
    if (pi < 0) return;
    __shared__ u64 sm[ROWS * kR16Row];
    const PrimeC P = primes[pi];
    const ulonglong2 *twp = tw + (size_t)pi * 65536;
    const int row0 = blockIdx.x * ROWS;
    u64 *d = bt.dst + ((size_t)row * bt.dst_stride + col) * 65536 + (size_t)row0 * 256;
    const ulonglong2 *rows = tw_rows + (size_t)pi * 256 * 15 * 16;
    if (P.q < (1ull << 47)) fwd_b16_body<true, OD>(d, twp, rows, row0, P, sm);
    else fwd_b16_body<false, OD>(d, twp, rows, row0, P, sm);
}

template <bool LAZY, bool OD>
__device__ __forceinline__ void inv_b16_body(const u64 *s, u64 *d, const ulonglong2 *twp,
                                             const ulonglong2 *rows, int row0, u64 q, u64 *sm)
{
    const int t = threadIdx.x, j = t & 15, r = t >> 4;
    constexpr int S1 = 8;
    const u64 q2 = 2 * q;
    u64 v[16];
    const int grow = row0 + r;
    const ulonglong2 *in = reinterpret_cast<const ulonglong2 *>(s + (size_t)r * 256 + 16 * j);
#pragma unroll
    for (int m = 0; m < 16; m += 2) {
        const ulonglong2 a = in[m / 2];
        v[m] = a.x;
        v[m + 1] = a.y;
    }
    gs16<LAZY>(v, twiddles<OD>([&](int st, int g) { return rows[((size_t)grow * 15 + (1 << st) - 1 + g) * 16 + j]; }),
               q, q2, 0);
    u64 *srow = sm + r * kR16Row;
#pragma unroll
    for (int m = 0; m < 16; m++) srow[pad16(16 * j + m)] = v[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 16; m++) v[m] = srow[pad16(j + 16 * m)];
    gs16<LAZY>(v, twiddles<OD>([&](int st, int g) { return twp[(1 << (S1 + st)) + (grow << st) + g]; }), q, q2, 4);
    u64 *drow = d + (size_t)r * 256;
#pragma unroll
    for (int m = 0; m < 16; m++) drow[j + 16 * m] = v[m];   // lazy (< 2^9 q or < 2q)
}

template <int ROWS, bool OD>
__global__ void __launch_bounds__(16 * ROWS, (OD ? 64 : 48) / ROWS)
ntt16_inv_b(const Batch bt, const PrimeC *__restrict__ primes, const ulonglong2 *__restrict__ itw,
            const ulonglong2 *__restrict__ itw_rows)
{
    const int limb = blockIdx.y;
    const int col = limb % bt.per_row, row = limb / bt.per_row;
    const int pi = bt.pidx[col];
    if (pi < 0) return;
    __shared__ u64 sm[ROWS * kR16Row];
    const u64 q = primes[pi].q;
    const ulonglong2 *twp = itw + (size_t)pi * 65536;
    const int row0 = blockIdx.x * ROWS;
    const u64 *s = bt.src + ((size_t)row * bt.src_stride + col) * 65536 + (size_t)row0 * 256;
    u64 *d = bt.dst + ((size_t)row * bt.dst_stride + col) * 65536 + (size_t)row0 * 256;
    const ulonglong2 *rows = itw_rows + (size_t)pi * 256 * 15 * 16;
    if (q < (1ull << 47)) inv_b16_body<true, OD>(s, d, twp, rows, row0, q, sm);
    else inv_b16_body<false, OD>(s, d, twp, rows, row0, q, sm);
}

template <bool LAZY, int COLS, bool OD>
__device__ __forceinline__ void inv_a16_body(u64 *d, const ulonglong2 *stw, u64 q, u64 ni, u64 nis,
                                             u64 *sm)
{
    const int t = threadIdx.x, c = t % COLS, r = t / COLS;
    constexpr int N2 = 256;
    const u64 q2 = 2 * q;
    u64 v[16];
#pragma unroll
    for (int m = 0; m < 16; m++) v[m] = d[(size_t)(16 * r + m) * N2 + c];
    gs16<LAZY>(v, twiddles<OD>([&](int st, int g) { return stw[(1 << (st + 4)) + (r << st) + g]; }), q, q2, 8);
#pragma unroll
    for (int m = 0; m < 16; m++) sm[(16 * r + m) * COLS + c] = v[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 16; m++) v[m] = sm[(r + 16 * m) * COLS + c];
    gs16<LAZY>(v, twiddles<OD>([&](int st, int g) { return stw[(1 << st) + g]; }), q, q2, 12);
#pragma unroll
    for (int m = 0; m < 16; m++) d[(size_t)(r + 16 * m) * N2 + c] = shoup_mul(v[m], ni, nis, q);
}

// col_scale (may be null): per limb column of the batch, a constant (and
// its Shoup companion) that replaces N^-1 in the final scaling
template <int COLS, bool OD>
__global__ void __launch_bounds__(16 * COLS, (OD ? 64 : 48) / COLS)
ntt16_inv_a(const Batch bt, const PrimeC *__restrict__ primes, const ulonglong2 *__restrict__ itw,
            const u64 *__restrict__ ninv, const u64 *__restrict__ col_scale)
{
    const int limb = blockIdx.y;
    const int col = limb % bt.per_row, row = limb / bt.per_row;
    const int pi = bt.pidx[col];
    if (pi < 0) return;
    __shared__ u64 sm[256 * COLS];
    __shared__ ulonglong2 stw[256];
    const u64 q = primes[pi].q;
    const ulonglong2 *twp = itw + (size_t)pi * 65536;
    for (int k = threadIdx.x; k < 256; k += blockDim.x) stw[k] = twp[k];
    __syncthreads();
    const int c0 = blockIdx.x * COLS;
    u64 *d = bt.dst + ((size_t)row * bt.dst_stride + col) * 65536 + c0;
    const u64 ni = col_scale ? col_scale[2 * col] : ninv[2 * pi];
    const u64 nis = col_scale ? col_scale[2 * col + 1] : ninv[2 * pi + 1];
    if (q < (1ull << 47)) inv_a16_body<true, COLS, OD>(d, stw, q, ni, nis, sm);
    else inv_a16_body<false, COLS, OD>(d, stw, q, ni, nis, sm);
}

// ModUp, N = 2^16: the base conversion of one digit to one output prime,
// fused into the first pass (column stages 0..7) of that output limb's
// forward NTT.  y: [ncol][nl][N], the conversion's inputs y_i = [x_i (D_j /
// q_i)^-1]_{q_i} in the coefficient domain (the inverse NTT of c1, scaled
// by modup_scale_tab); digits: [ncol][beta][E][N], pass-A output of every
// limb outside the digit (pass B follows as for any forward NTT).  Grid:
// (256 / COLS column tiles, output index t, column f x beta + digit).
template <int NMAX, int COLS, bool OD>
__global__ void __launch_bounds__(16 * COLS, (OD ? 64 : 48) / COLS)
k_modup_ntt16_a(const u64 *__restrict__ y, int nl, u64 *digits, int beta, int E,
                const ConvTab *__restrict__ tabs, const PrimeC *__restrict__ primes,
                const ulonglong2 *__restrict__ tw)
{
    const int f = blockIdx.z / beta, dg = blockIdx.z % beta, t = blockIdx.y;
    const ConvTab &T = tabs[dg];
    if (t >= T.n_out) return;
    __shared__ u64 sm[256 * COLS];
    __shared__ ulonglong2 stw[256];
    const int pi = T.out_p[t];
    const PrimeC P = primes[pi];
    const ulonglong2 *twp = tw + (size_t)pi * 65536;
    for (int k = threadIdx.x; k < 256; k += blockDim.x) stw[k] = twp[k];
    u64 hm_[NMAX];
    const u64 *src[NMAX];
#pragma unroll
    for (int k = 0; k < NMAX; k++) {
        hm_[k] = k < T.n_in ? T.hmod[k][t] : 0;
        src[k] = y + ((size_t)f * nl + (k < T.n_in ? T.in_l[k] : 0)) * 65536;
    }
    const int c = threadIdx.x % COLS, r = threadIdx.x / COLS, c0 = blockIdx.x * COLS;
    u64 v[16];
#pragma unroll
    for (int m = 0; m < 16; m++) {
        const size_t idx = (size_t)(r + 16 * m) * 256 + c0 + c;
        u64 a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
        for (int k = 0; k < NMAX; k++)
            if (k < T.n_in) mac_split(a0, a1, a2, split30(src[k][idx]), hm_[k]);
        u64 hi = 0, lo = 0;
        fold30(hi, lo, a0, a1, a2);
        v[m] = redc(hi, lo, P);
    }
    __syncthreads();   // stw
    u64 *d = digits + (((size_t)f * beta + dg) * E + T.out_l[t]) * 65536 + c0;
    if (P.q < (1ull << 47)) fwd_a16_rounds<true, COLS, OD>(v, d, stw, P.q, sm);
    else fwd_a16_rounds<false, COLS, OD>(v, d, stw, P.q, sm);
}

// Stages are taken two at a time (radix-4 rounds: four elements, four
// butterflies, one shared-memory round trip and one barrier per two
// stages).  Within a sub-transform of 2^LS elements, a round on stages
// (s, s+1) (s counted inside the sub-transform) works on element groups
// {r, r + h/2, r + h, r + 3h/2} with h = 2^(LS-s-1), r = (i << (LS-s)) + j,
// i = unit >> (LS-s-2), j = unit & (h/2 - 1); stage s uses twiddle index
// 2^s + i, stage s+1 uses 2^(s+1) + 2i and 2^(s+1) + 2i + 1 (offset by the
// sub-transform's position in the global stage numbering, see callers).

template <int LOGN>
__global__ void __launch_bounds__(kNttThreads)
ntt_fwd_a(const Batch bt, const PrimeC *__restrict__ primes, const ulonglong2 *__restrict__ tw)
{
    constexpr int S1 = LOGN / 2, N = 1 << LOGN, N1 = 1 << S1, N2 = N >> S1;
    constexpr int LC = 4;   // log2 kColsA
    const int limb = blockIdx.y;
    const int col = limb % bt.per_row, row = limb / bt.per_row;
    const int pi = bt.pidx[col];
    if (pi < 0) return;
    extern __shared__ u64 sm[];
    ulonglong2 *stw = reinterpret_cast<ulonglong2 *>(sm + N1 * kColsA);
    const u64 q = primes[pi].q, q2 = 2 * q;
    const ulonglong2 *twp = tw + (size_t)pi * N;
    const u64 *src = bt.src + ((size_t)row * bt.src_stride + col) * N;
    u64 *dst = bt.dst + ((size_t)row * bt.dst_stride + col) * N;
    const int c0 = blockIdx.x * kColsA;
    for (int i = threadIdx.x; i < N1; i += kNttThreads) stw[i] = twp[i];
    for (int idx = threadIdx.x; idx < N1 * kColsA; idx += kNttThreads)
        sm[idx] = src[(size_t)(idx >> LC) * N2 + c0 + (idx & (kColsA - 1))];
    __syncthreads();
    int s = 0;
#pragma unroll
    for (; s + 1 < S1; s += 2) {
        const int lq = S1 - s - 2;   // log of h/2
#pragma unroll 2
        for (int b = threadIdx.x; b < (N1 / 4) * kColsA; b += kNttThreads) {
            const int c = b & (kColsA - 1), u = b >> LC;
            const int i = u >> lq, j = u & ((1 << lq) - 1);
            const int r = (i << (lq + 2)) + j;
            const ulonglong2 w1 = stw[(1 << s) + i];
            const ulonglong2 w2 = stw[(2 << s) + 2 * i], w3 = stw[(2 << s) + 2 * i + 1];
            u64 *p0 = sm + r * kColsA + c;
            const int dq = (1 << lq) * kColsA;
            u64 a0 = p0[0], a1 = p0[dq], a2 = p0[2 * dq], a3 = p0[3 * dq];
            ct_bfly(a0, a2, w1, q, q2);
            ct_bfly(a1, a3, w1, q, q2);
            ct_bfly(a0, a1, w2, q, q2);
            ct_bfly(a2, a3, w3, q, q2);
            p0[0] = a0;
            p0[dq] = a1;
            p0[2 * dq] = a2;
            p0[3 * dq] = a3;
        }
        __syncthreads();
    }
    if (s < S1) {   // odd stage count: last radix-2 stage (h = 1)
        for (int b = threadIdx.x; b < (N1 / 2) * kColsA; b += kNttThreads) {
            const int c = b & (kColsA - 1), i = b >> LC;
            u64 *p0 = sm + (2 * i) * kColsA + c;
            u64 a0 = p0[0], a1 = p0[kColsA];
            ct_bfly(a0, a1, stw[(1 << s) + i], q, q2);
            p0[0] = a0;
            p0[kColsA] = a1;
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < N1 * kColsA; idx += kNttThreads)
        dst[(size_t)(idx >> LC) * N2 + c0 + (idx & (kColsA - 1))] = sm[idx];   // lazy, < 4q
}

template <int LOGN>
__global__ void __launch_bounds__(kNttThreads)
ntt_fwd_b(const Batch bt, const PrimeC *__restrict__ primes, const ulonglong2 *__restrict__ tw)
{
    constexpr int S1 = LOGN / 2, N = 1 << LOGN, N1 = 1 << S1, LN2 = LOGN - S1, N2 = 1 << LN2;
    constexpr int R = (kElemsB / N2) < N1 ? (kElemsB / N2) : N1;
    const int limb = blockIdx.y;
    const int col = limb % bt.per_row, row = limb / bt.per_row;
    const int pi = bt.pidx[col];
    if (pi < 0) return;
    extern __shared__ u64 sm[];
    const u64 q = primes[pi].q, q2 = 2 * q;
    const ulonglong2 *twp = tw + (size_t)pi * N;
    const int row0 = blockIdx.x * R;
    u64 *d = bt.dst + ((size_t)row * bt.dst_stride + col) * N + (size_t)row0 * N2;
    for (int idx = threadIdx.x; idx < R * N2; idx += kNttThreads) sm[idx] = d[idx];
    __syncthreads();
    int ls = 0;   // stage inside the row; global stage S1 + ls
#pragma unroll
    for (; ls + 1 < LN2; ls += 2) {
        const int s = S1 + ls;
        const int lq = LN2 - ls - 2;
#pragma unroll 2
        for (int b = threadIdx.x; b < R * (N2 / 4); b += kNttThreads) {
            const int r = b >> (LN2 - 2), u = b & (N2 / 4 - 1);
            const int i = u >> lq, j = u & ((1 << lq) - 1);
            const int pos = (i << (lq + 2)) + j;
            const int gi = ((row0 + r) << ls) + i;
            const ulonglong2 w1 = twp[(1 << s) + gi];
            const ulonglong2 w2 = twp[(2 << s) + 2 * gi], w3 = twp[(2 << s) + 2 * gi + 1];
            u64 *p0 = sm + r * N2 + pos;
            const int dq = 1 << lq;
            u64 a0 = p0[0], a1 = p0[dq], a2 = p0[2 * dq], a3 = p0[3 * dq];
            ct_bfly(a0, a2, w1, q, q2);
            ct_bfly(a1, a3, w1, q, q2);
            ct_bfly(a0, a1, w2, q, q2);
            ct_bfly(a2, a3, w3, q, q2);
            p0[0] = a0;
            p0[dq] = a1;
            p0[2 * dq] = a2;
            p0[3 * dq] = a3;
        }
        __syncthreads();
    }
    if (ls < LN2) {   // last radix-2 stage, half distance 1
        const int s = S1 + ls;
        for (int b = threadIdx.x; b < R * (N2 / 2); b += kNttThreads) {
            const int r = b >> (LN2 - 1), i = b & (N2 / 2 - 1);
            u64 *p0 = sm + r * N2 + 2 * i;
            u64 a0 = p0[0], a1 = p0[1];
            ct_bfly(a0, a1, twp[(1 << s) + ((row0 + r) << ls) + i], q, q2);
            p0[0] = a0;
            p0[1] = a1;
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < R * N2; idx += kNttThreads) d[idx] = reduce4(sm[idx], q);
}

template <int LOGN>
__global__ void __launch_bounds__(kNttThreads)
ntt_inv_b(const Batch bt, const PrimeC *__restrict__ primes, const ulonglong2 *__restrict__ itw)
{
    constexpr int S1 = LOGN / 2, N = 1 << LOGN, N1 = 1 << S1, LN2 = LOGN - S1, N2 = 1 << LN2;
    constexpr int R = (kElemsB / N2) < N1 ? (kElemsB / N2) : N1;
    const int limb = blockIdx.y;
    const int col = limb % bt.per_row, row = limb / bt.per_row;
    const int pi = bt.pidx[col];
    if (pi < 0) return;
    extern __shared__ u64 sm[];
    const u64 q = primes[pi].q, q2 = 2 * q;
    const ulonglong2 *twp = itw + (size_t)pi * N;
    const int row0 = blockIdx.x * R;
    const u64 *sr = bt.src + ((size_t)row * bt.src_stride + col) * N + (size_t)row0 * N2;
    u64 *d = bt.dst + ((size_t)row * bt.dst_stride + col) * N + (size_t)row0 * N2;
    for (int idx = threadIdx.x; idx < R * N2; idx += kNttThreads) sm[idx] = sr[idx];
    __syncthreads();
    int ls = LN2 - 1;
    if (LN2 & 1) {   // odd: the last stage (half distance 1) alone first
        const int s = S1 + ls;
        for (int b = threadIdx.x; b < R * (N2 / 2); b += kNttThreads) {
            const int r = b >> (LN2 - 1), i = b & (N2 / 2 - 1);
            u64 *p0 = sm + r * N2 + 2 * i;
            u64 a0 = p0[0], a1 = p0[1];
            gs_bfly(a0, a1, twp[(1 << s) + ((row0 + r) << ls) + i], q, q2);
            p0[0] = a0;
            p0[1] = a1;
        }
        __syncthreads();
        ls--;
    }
#pragma unroll
    for (; ls >= 1; ls -= 2) {   // stages (ls-1, ls), higher one first
        const int lo = ls - 1, s = S1 + lo;
        const int lq = LN2 - lo - 2;
#pragma unroll 2
        for (int b = threadIdx.x; b < R * (N2 / 4); b += kNttThreads) {
            const int r = b >> (LN2 - 2), u = b & (N2 / 4 - 1);
            const int i = u >> lq, j = u & ((1 << lq) - 1);
            const int pos = (i << (lq + 2)) + j;
            const int gi = ((row0 + r) << lo) + i;
            const ulonglong2 w1 = twp[(1 << s) + gi];
            const ulonglong2 w2 = twp[(2 << s) + 2 * gi], w3 = twp[(2 << s) + 2 * gi + 1];
            u64 *p0 = sm + r * N2 + pos;
            const int dq = 1 << lq;
            u64 a0 = p0[0], a1 = p0[dq], a2 = p0[2 * dq], a3 = p0[3 * dq];
            gs_bfly(a0, a1, w2, q, q2);
            gs_bfly(a2, a3, w3, q, q2);
            gs_bfly(a0, a2, w1, q, q2);
            gs_bfly(a1, a3, w1, q, q2);
            p0[0] = a0;
            p0[dq] = a1;
            p0[2 * dq] = a2;
            p0[3 * dq] = a3;
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < R * N2; idx += kNttThreads) d[idx] = sm[idx];   // < 2q
}

template <int LOGN>
__global__ void __launch_bounds__(kNttThreads)
ntt_inv_a(const Batch bt, const PrimeC *__restrict__ primes, const ulonglong2 *__restrict__ itw,
          const u64 *__restrict__ ninv)
{
    constexpr int S1 = LOGN / 2, N = 1 << LOGN, N1 = 1 << S1, N2 = N >> S1;
    constexpr int LC = 4;
    const int limb = blockIdx.y;
    const int col = limb % bt.per_row, row = limb / bt.per_row;
    const int pi = bt.pidx[col];
    if (pi < 0) return;
    extern __shared__ u64 sm[];
    ulonglong2 *stw = reinterpret_cast<ulonglong2 *>(sm + N1 * kColsA);
    const u64 q = primes[pi].q, q2 = 2 * q;
    const ulonglong2 *twp = itw + (size_t)pi * N;
    u64 *d = bt.dst + ((size_t)row * bt.dst_stride + col) * N;
    const int c0 = blockIdx.x * kColsA;
    for (int i = threadIdx.x; i < N1; i += kNttThreads) stw[i] = twp[i];
    for (int idx = threadIdx.x; idx < N1 * kColsA; idx += kNttThreads)
        sm[idx] = d[(size_t)(idx >> LC) * N2 + c0 + (idx & (kColsA - 1))];
    __syncthreads();
    int s = S1 - 1;
    if (S1 & 1) {   // odd: last stage (h = 1) alone first
        for (int b = threadIdx.x; b < (N1 / 2) * kColsA; b += kNttThreads) {
            const int c = b & (kColsA - 1), i = b >> LC;
            u64 *p0 = sm + (2 * i) * kColsA + c;
            u64 a0 = p0[0], a1 = p0[kColsA];
            gs_bfly(a0, a1, stw[(1 << s) + i], q, q2);
            p0[0] = a0;
            p0[kColsA] = a1;
        }
        __syncthreads();
        s--;
    }
#pragma unroll
    for (; s >= 1; s -= 2) {   // stages (s-1, s), higher one first
        const int lo = s - 1;
        const int lq = S1 - lo - 2;
#pragma unroll 2
        for (int b = threadIdx.x; b < (N1 / 4) * kColsA; b += kNttThreads) {
            const int c = b & (kColsA - 1), u = b >> LC;
            const int i = u >> lq, j = u & ((1 << lq) - 1);
            const int r = (i << (lq + 2)) + j;
            const ulonglong2 w1 = stw[(1 << lo) + i];
            const ulonglong2 w2 = stw[(2 << lo) + 2 * i], w3 = stw[(2 << lo) + 2 * i + 1];
            u64 *p0 = sm + r * kColsA + c;
            const int dq = (1 << lq) * kColsA;
            u64 a0 = p0[0], a1 = p0[dq], a2 = p0[2 * dq], a3 = p0[3 * dq];
            gs_bfly(a0, a1, w2, q, q2);
            gs_bfly(a2, a3, w3, q, q2);
            gs_bfly(a0, a2, w1, q, q2);
            gs_bfly(a1, a3, w1, q, q2);
            p0[0] = a0;
            p0[dq] = a1;
            p0[2 * dq] = a2;
            p0[3 * dq] = a3;
        }
        __syncthreads();
    }
    const u64 ni = ninv[2 * pi], nis = ninv[2 * pi + 1];
    for (int idx = threadIdx.x; idx < N1 * kColsA; idx += kNttThreads)
        d[(size_t)(idx >> LC) * N2 + c0 + (idx & (kColsA - 1))] = shoup_mul(sm[idx], ni, nis, q);
}

// ------------------------------------------------------------------------
// element-wise kernels over a Batch (grid: x blocks, limbs)
// ------------------------------------------------------------------------
__device__ __forceinline__ const u64 *limb_ptr(const u64 *base, int stride, int per_row, int limb,
                                               int N)
{
    return base + ((size_t)(limb / per_row) * stride + (limb % per_row)) * N;
}

__global__ void k_to_mont(const Batch bt, const PrimeC *__restrict__ primes, int N)
{
    const int limb = blockIdx.y;
    const int pi = bt.pidx[limb % bt.per_row];
    if (pi < 0) return;
    const PrimeC P = primes[pi];
    u64 *d = const_cast<u64 *>(limb_ptr(bt.dst, bt.dst_stride, bt.per_row, limb, N));
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x)
        d[x] = mont_mul(d[x], P.r2, P);
}

__global__ void k_from_mont(const Batch bt, const PrimeC *__restrict__ primes, int N)
{
    const int limb = blockIdx.y;
    const int pi = bt.pidx[limb % bt.per_row];
    if (pi < 0) return;
    const PrimeC P = primes[pi];
    u64 *d = const_cast<u64 *>(limb_ptr(bt.dst, bt.dst_stride, bt.per_row, limb, N));
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x)
        d[x] = redc(0, d[x], P);
}

// c = a * b (both plain NTT-domain values)
__global__ void k_pointwise(const u64 *a, const u64 *b, u64 *c, const Batch bt,
                            const PrimeC *__restrict__ primes, int N)
{
    const int limb = blockIdx.y;
    const int pi = bt.pidx[limb % bt.per_row];
    if (pi < 0) return;
    const PrimeC P = primes[pi];
    const size_t off = (size_t)limb * N;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x)
        c[off + x] = mont_mul(mont_mul(a[off + x], b[off + x], P), P.r2, P);
}

__global__ void k_add(const u64 *a, const u64 *b, u64 *c, const Batch bt,
                      const PrimeC *__restrict__ primes, int N)
{
    const int limb = blockIdx.y;
    const int pi = bt.pidx[limb % bt.per_row];
    if (pi < 0) return;
    const u64 q = primes[pi].q;
    const size_t off = (size_t)limb * N;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x)
        c[off + x] = add_mod(a[off + x], b[off + x], q);
}

__global__ void k_neg(const u64 *a, u64 *c, const Batch bt, const PrimeC *__restrict__ primes,
                      int N)
{
    const int limb = blockIdx.y;
    const int pi = bt.pidx[limb % bt.per_row];
    if (pi < 0) return;
    const u64 q = primes[pi].q;
    const size_t off = (size_t)limb * N;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x) {
        u64 v = a[off + x];
        c[off + x] = v ? q - v : 0;
    }
}

// c = a * s_limb (scalar per limb column, Shoup), s given as (w, w') pairs
__global__ void k_scalar(const u64 *a, u64 *c, const Batch bt, const PrimeC *__restrict__ primes,
                         const u64 *__restrict__ scal, int N)
{
    const int limb = blockIdx.y;
    const int col = limb % bt.per_row;
    const int pi = bt.pidx[col];
    if (pi < 0) return;
    const u64 q = primes[pi].q, w = scal[2 * col], ws = scal[2 * col + 1];
    const size_t off = (size_t)limb * N;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x)
        c[off + x] = shoup_mul(a[off + x], w, ws, q);
}

// automorphism X -> X^g in the bit-reversed NTT order:
// out[j] = a[brv(((2 brv(j) + 1) g mod 2N - 1) / 2)]
__device__ __forceinline__ int auto_src(int j, uint32_t g, int log_n)
{
    uint32_t r = __brev((uint32_t)j) >> (32 - log_n);
    uint32_t e = ((2 * r + 1) * g) & ((2u << log_n) - 1);
    return (int)(__brev((e - 1) >> 1) >> (32 - log_n));
}

__global__ void k_automorphism(const u64 *a, u64 *c, int nlimbs, uint32_t g, int log_n)
{
    const int N = 1 << log_n;
    const size_t off = (size_t)blockIdx.y * N;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x)
        c[off + x] = a[off + auto_src(x, g, log_n)];
}

// small signed coefficients -> residues of each listed prime
__global__ void k_small_to_res(const int8_t *e, u64 *out, const int *pidx, const PrimeC *primes,
                               int N)
{
    const int limb = blockIdx.y;
    const u64 q = primes[pidx[limb]].q;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x) {
        int v = e[x];
        out[(size_t)limb * N + x] = v < 0 ? q - (u64)(-v) : (u64)v;
    }
}

// SplitMix64's output function (Steele, Lea and Flood, OOPSLA 2014)
__device__ __forceinline__ u64 sm_mix_dev(u64 z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// The uniform part of seeded ciphertexts: column c is ciphertext index0 + c,
// whose stream (seed, purpose, index) starts from s0 = mix(seed ^ (purpose
// << 48) ^ index) and has word j = mix(s0 + (j + 1) gamma); coefficient x of
// limb i is (w_hi 2^64 + w_lo) mod q_i with w_lo, w_hi the words 2(i N + x)
// and 2(i N + x) + 1.  [w_hi]_q 2^64 mod q is the Montgomery product of
// [w_hi]_q with R^2 mod q (R = 2^64).  Ciphertext c is written at ct + c *
// ct_pitch: its uniform part at offset nl N, and, when c0 is given, its c0
// copied from c0 + c * nl N.
__global__ void k_expand_uniform(u64 *ct, size_t ct_pitch, const u64 *__restrict__ c0, int nl, u64 seed,
                                 u64 purpose, u64 index0, const PrimeC *__restrict__ primes, int N)
{
    const int i = blockIdx.y, c = blockIdx.z;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    const PrimeC P = primes[i];
    const u64 gamma = 0x9E3779B97F4A7C15ull;
    const u64 s0 = sm_mix_dev(seed ^ (purpose << 48) ^ (index0 + (u64)c));
    const u64 j = 2 * ((u64)i * (u64)N + (u64)x);
    const u64 lo = sm_mix_dev(s0 + (j + 1) * gamma), hi = sm_mix_dev(s0 + (j + 2) * gamma);
    const u64 h = mont_mul(reduce_word(hi, P), P.r2, P);
    u64 *o = ct + (size_t)c * ct_pitch + (size_t)i * N + x;
    o[(size_t)nl * N] = add_mod(h, reduce_word(lo, P), P.q);
    if (c0) *o = c0[((size_t)c * nl + i) * N + x];
}

__global__ void k_copy_limbs(const u64 *src, int src_ls, u64 *dst, int dst_ls, int nl, int N)
{
    const int poly = blockIdx.z, i = blockIdx.y;
    const u64 *s = src + ((size_t)poly * src_ls + i) * N;
    u64 *d = dst + ((size_t)poly * dst_ls + i) * N;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x)
        d[x] = s[x];
}

// ------------------------------------------------------------------------
// combination: Z[j][p][i] = sum_f c[i][f][j] * X[f][p][i]   (coefficient domain)
// constants in Montgomery form, one Montgomery reduction at the end.  For
// primes below 2^46 the products are 23-bit split sums (mac_split); for the
// others 128-bit sums with the high word folded mod q every chunk.
// ------------------------------------------------------------------------
constexpr int kCombJ = 8;
constexpr int kCombChunk = 128;

// Columns fb..fe-1 of X; with accumulate set, the result is added to Z.
// The nj = ceil(Fp / kCombJ) output blocks of one slot range are
// neighbouring CTAs (blockIdx.x = slot block * nj + output block), so they
// run together and the later ones find the input words in L2: X is read from
// HBM once for all F' outputs.
__global__ void __launch_bounds__(256)
k_comb(const u64 *__restrict__ X, int F, int fb, int fe, int accumulate, int Fp, int nj, int level,
       const u64 *__restrict__ consts, u64 *Z, int z_ls, const PrimeC *__restrict__ primes,
       int N)
{
    __shared__ u64 cs[kCombChunk][kCombJ];
    const int i = blockIdx.y, p = blockIdx.z;
    const int j0 = (blockIdx.x % nj) * kCombJ;
    const int x = (blockIdx.x / nj) * blockDim.x + threadIdx.x;
    const PrimeC P = primes[i];
    const bool split = P.q < (1ull << 46);
    const int nl = level + 1;
    u64 a0[kCombJ], a1[kCombJ], a2[kCombJ];   // split: A0, A1, A2; else lo, hi, unused
#pragma unroll
    for (int j = 0; j < kCombJ; j++) a0[j] = a1[j] = a2[j] = 0;
    for (int f0 = fb; f0 < fe; f0 += kCombChunk) {
        const int fc = min(kCombChunk, fe - f0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < kCombChunk * kCombJ; idx += blockDim.x) {
            int ff = idx / kCombJ, jj = idx % kCombJ;
            const u64 c = (ff < fc && j0 + jj < Fp) ? consts[((size_t)i * F + f0 + ff) * Fp + j0 + jj] : 0;
            cs[ff][jj] = split ? split23(c) : c;
        }
        __syncthreads();
        if (x < N) {
            if (split) {
                for (int ff = 0; ff < fc; ff++) {
                    const u64 xv = split23(X[(((size_t)(f0 + ff) * 2 + p) * nl + i) * N + x]);
#pragma unroll
                    for (int j = 0; j < kCombJ; j++) mac_split(a0[j], a1[j], a2[j], xv, cs[ff][j]);
                }
            } else {
                for (int ff = 0; ff < fc; ff++) {
                    const u64 xv = X[(((size_t)(f0 + ff) * 2 + p) * nl + i) * N + x];
#pragma unroll
                    for (int j = 0; j < kCombJ; j++) mac128(a1[j], a0[j], xv, cs[ff][j]);
                }
#pragma unroll
                for (int j = 0; j < kCombJ; j++) a1[j] = reduce_word(a1[j], P);
            }
        }
    }
    if (x < N) {
#pragma unroll
        for (int j = 0; j < kCombJ; j++)
            if (j0 + j < Fp) {
                u64 *z = Z + (((size_t)(j0 + j) * 2 + p) * z_ls + i) * N + x;
                const u64 r = split ? fold_split(a0[j], a1[j], a2[j], P) : redc(a1[j], a0[j], P);
                *z = accumulate ? add_mod(*z, r, P.q) : r;
            }
    }
}

// ------------------------------------------------------------------------
// rescale
// ------------------------------------------------------------------------
// Rescale rounds: c <- floor((c + h) / q_l), h = (q_l - 1) / 2, so the
// error of every coefficient is centred (a floor biases all of them by -1/2,
// and decryption amplifies that bias at the slots near 1).  Per limb:
//   out_i = (in_i + [h]_{q_i} - [r]_{q_i}) * q_l^-1,  r = [in_l + h]_{q_l}.
// coefficient domain
__global__ void k_rescale_coef(const u64 *in, int in_ls, u64 *out, int out_ls, int level,
                               const PrimeC *__restrict__ primes, const u64 *__restrict__ tab,
                               int N)
{
    const int i = blockIdx.y, poly = blockIdx.z;
    const PrimeC P = primes[i], Pl = primes[level];
    const u64 inv = tab[2 * i], invs = tab[2 * i + 1];
    const u64 h = Pl.q >> 1, hi = reduce_word(h, P);
    const u64 *top = in + ((size_t)poly * in_ls + level) * N;
    const u64 *src = in + ((size_t)poly * in_ls + i) * N;
    u64 *dst = out + ((size_t)poly * out_ls + i) * N;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x) {
        const u64 r = reduce_word(reduce_word(top[x], Pl) + h, Pl);
        dst[x] = shoup_mul(sub_mod(add_mod(src[x], hi, P.q), reduce_word(r, P), P.q), inv, invs, P.q);
    }
}

// the top limb l (coefficient domain, one per poly) -> [r]_{q_i} - [h]_{q_i}
// for i < level, r = [c_l + h]_{q_l}: what the rounded rescale subtracts
// (after its NTT) from limb i
__global__ void k_bcast_reduce(const u64 *r, int r_ls, int r_limb, u64 *out, int level,
                               const PrimeC *__restrict__ primes, int N)
{
    const int i = blockIdx.y, poly = blockIdx.z;
    const PrimeC P = primes[i], Pl = primes[r_limb];
    const u64 h = Pl.q >> 1, hi = reduce_word(h, P);
    const u64 *src = r + ((size_t)poly * r_ls + r_limb) * N;
    u64 *dst = out + ((size_t)poly * level + i) * N;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x) {
        const u64 t = reduce_word(reduce_word(src[x], Pl) + h, Pl);
        dst[x] = sub_mod(reduce_word(t, P), hi, P.q);
    }
}

// NTT domain finish: ct_i = (ct_i - r_i) * q_l^-1
__global__ void k_rescale_finish(u64 *ct, int ls, const u64 *rr, int level,
                                 const PrimeC *__restrict__ primes, const u64 *__restrict__ tab,
                                 int N)
{
    const int i = blockIdx.y, poly = blockIdx.z;
    const u64 q = primes[i].q, inv = tab[2 * i], invs = tab[2 * i + 1];
    u64 *c = ct + ((size_t)poly * ls + i) * N;
    const u64 *r = rr + ((size_t)poly * level + i) * N;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x)
        c[x] = shoup_mul(sub_mod(c[x], r[x], q), inv, invs, q);
}


// ------------------------------------------------------------------------
// base conversion (approximate, no overflow correction):
//   out_p = sum_k [x_k * (B/b_k)^-1]_{b_k} * (B/b_k) mod p
// y_k in [0, b_k), (B/b_k) mod p in Montgomery form, n_in <= 8 products of
// two words below 2^61 accumulate below p * 2^64, so one Montgomery
// reduction gives the exact residue.
// ------------------------------------------------------------------------
// NMAX bounds T.n_in at compile time, so that y stays in registers.  y and
// the table hold 30-bit halves: at most 8 products per partial sum, and the
// total below 8 2^60 p keeps its high word below p for the Montgomery step.
template <int NMAX>
__device__ __forceinline__ u64 conv_point(const ConvTab &T, const u64 *y, int t, const PrimeC &P,
                                          int c = 0)
{
    static_assert(NMAX <= 8, "at most 8 inputs per conversion");
    u64 a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
    for (int k = 0; k < NMAX; k++)
        if (k < T.n_in) mac_split(a0, a1, a2, y[k], T.hmod[k][t]);
    // centred conversion: c B subtracted (c <= 7: the product adds below
    // 2^34 to the partial sums, within the 8-term bound for K <= 7)
    if (c) mac_split(a0, a1, a2, (u64)c, T.negb[t]);
    u64 hi = 0, lo = 0;
    fold30(hi, lo, a0, a1, a2);
    return redc(hi, lo, P);
}

// returns the number of inputs y_k above b_k / 2: taking those as y_k - b_k
// centres the conversion (see k_moddown_conv)
template <int NMAX>
__device__ __forceinline__ int conv_inputs(const ConvTab &T, const u64 *src, size_t limb_stride,
                                           u64 *y, const PrimeC *__restrict__ primes)
{
    int c = 0;
#pragma unroll
    for (int k = 0; k < NMAX; k++)
        if (k < T.n_in) {
            const u64 v = src[(size_t)T.in_l[k] * limb_stride];
            const u64 b = primes[T.in_p[k]].q;
            const u64 yk = shoup_mul(v, T.hinv[k], T.hinv_s[k], b);
            c += yk > (b >> 1);
            y[k] = split30(yk);
        }
    return c;
}

// ModUp conversion.  c1c: [ncol][nl][N] coefficient domain (nl = level+1);
// digits: [ncol][beta][E][N]; writes every limb outside digit dg.
template <int NMAX>
__global__ void __launch_bounds__(256)
k_modup_conv(const u64 *__restrict__ c1c, int nl, u64 *digits, int beta, int E,
             const ConvTab *__restrict__ tabs, const PrimeC *__restrict__ primes, int N)
{
    const int f = blockIdx.z / beta, dg = blockIdx.z % beta;
    const ConvTab &T = tabs[dg];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    u64 y[NMAX];
    conv_inputs<NMAX>(T, c1c + (size_t)f * nl * N + x, N, y, primes);
    u64 *out = digits + ((size_t)f * beta + dg) * E * N;
    for (int t = 0; t < T.n_out; t++) {
        const PrimeC P = primes[T.out_p[t]];
        out[(size_t)T.out_l[t] * N + x] = conv_point<NMAX>(T, y, t, P);
    }
}

// ModDown conversion P -> q_0..q_level.  u: [npoly][E][N] (P limbs in the
// coefficient domain at positions level+1..), conv: [npoly][level+1][N].
// The ModDown's conversion is centred: y_k = [u_k (P/p_k)^-1]_{p_k} taken
// in (-p_k/2, p_k/2], i.e. the plain conversion minus c P with c the number
// of y_k above p_k/2.  Then (u - Conv)/P differs from u/P by minus
// sum_k y_k / p_k, which has mean zero; the plain conversion (y_k in
// [0, p_k)) biases every coefficient by -K/2, and in c1 decryption
// multiplies that bias by s and amplifies it at the slots near 1.
template <int NMAX>
__global__ void __launch_bounds__(256)
k_moddown_conv(const u64 *__restrict__ u, int E, u64 *conv, int nl,
               const ConvTab *__restrict__ tab, const PrimeC *__restrict__ primes, int N)
{
    const int poly = blockIdx.y;
    const ConvTab &T = *tab;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    u64 y[NMAX];
    const int c = conv_inputs<NMAX>(T, u + (size_t)poly * E * N + x, N, y, primes);
    for (int t = 0; t < T.n_out; t++) {
        const PrimeC P = primes[T.out_p[t]];
        conv[((size_t)poly * nl + T.out_l[t]) * N + x] = conv_point<NMAX>(T, y, t, P, c);
    }
}

// ------------------------------------------------------------------------
// key switching inner product with the automorphism folded into the gather:
//   u_p[f][i][x] = sum_d D_d[f][i][sigma_g(x)] * evk_g[d][p][i][x]
// D_d limb i is the lane's own c1 limb when i belongs to digit d, else the
// ModUp output.  The key (Montgomery form, [beta_L][2][nq+np][N]) is read
// once per (x, i) and reused for every column.
// ------------------------------------------------------------------------
constexpr int kMaxBeta = 16;   // beta * p^2 < p * 2^64 needs beta * p < 2^64: p < 2^60

// Each thread owns two adjacent slots x, x+1 (16-byte accesses).  In the
// bit-reversed NTT order the automorphism maps every aligned pair {x, x+1}
// onto an aligned pair {2m, 2m+1}, so the gather is one 16-byte load plus a
// swap when sigma(x) is odd.
__device__ __forceinline__ ulonglong2 gather_pair(const u64 *limb, int m2, bool swap)
{
    const ulonglong2 v = reinterpret_cast<const ulonglong2 *>(limb)[m2 >> 1];
    return swap ? make_ulonglong2(v.y, v.x) : v;
}

// Several rotations of one lane in one launch: blockIdx.y picks the rotation
// and blockIdx.z the limb, so the CTAs of one limb run together and the
// lane's digits of that limb (ncol * beta limbs) are read from HBM once and
// gathered again from L2 by the other rotations.
constexpr int kKsMulti = 24;
struct KsSet {
    int n;
    const u64 *key[kKsMulti];
    uint32_t g[kKsMulti];
    u64 *u[kKsMulti];
};

// With pmodq given, part 0 also receives P phi_g(c0) on the limbs of Q
// (P mod q_i and its Shoup companion at pmodq[2i], pmodq[2i+1]), so that
// ModDown of u is Rot(c) itself: ModDown(A + P B) = ModDown(A) + B exactly.
// LESS: CTAs per SM one fewer than the default bound (more registers per
// thread, fewer spills, lower occupancy); a tuning choice of the batched form.
constexpr int ks_min_blocks(int beta, int less)
{
    return (beta <= 4 ? 4 : beta <= 5 ? 3 : 2) - less > 0 ? (beta <= 4 ? 4 : beta <= 5 ? 3 : 2) - less : 1;
}

// KSM: the thread's split key words are parked in shared memory (its own
// 2 x BETA entries, no sharing, so no barrier) instead of registers, which
// frees about 40 registers for one more CTA per SM; a tuning choice.
template <int BETA, int LESS, bool KSM>
__global__ void __launch_bounds__(256, KSM ? (BETA <= 4 ? 5 : 4) : ks_min_blocks(BETA, LESS))
k_ks_ip(const KsSet ks, int KL, const u64 *__restrict__ lane, int ls,
        const u64 *__restrict__ digits, int ncol, int level, int E, int alpha, int nq,
        int log_n, const PrimeC *__restrict__ primes, const u64 *__restrict__ pmodq)
{
    extern __shared__ ulonglong2 kpark[];   // KSM: [BETA][2][blockDim.x]
    const int N = 1 << log_n;
    const int rot = blockIdx.y, i = blockIdx.z;
    const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= N) return;
    const u64 *key = ks.key[rot];
    u64 *u = ks.u[rot];
    const int pi = i <= level ? i : nq + (i - level - 1);
    const PrimeC P = primes[pi];
    const int sx = auto_src(x, ks.g[rot], log_n);
    const bool swap = sx & 1;
    const int own = i <= level ? i / alpha : -1;
    // Sums of BETA products of words below 2^60: with 30-bit halves (keys
    // split once per thread, each gathered digit word once for its two
    // products) the three 64-bit partial sums hold up to 8 products per
    // term; more digits take the 128-bit sums.  The total, below
    // BETA 2^60 q, keeps its high word below q for the Montgomery step.
    constexpr bool SPLIT = BETA <= 8;
    ulonglong2 kb[KSM ? 1 : BETA], ka[KSM ? 1 : BETA];
#pragma unroll
    for (int d = 0; d < BETA; d++) {
        ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(key + (((size_t)d * 2 + 0) * KL + pi) * N + x);
        ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(key + (((size_t)d * 2 + 1) * KL + pi) * N + x);
        if (SPLIT) {
            b = make_ulonglong2(split30(b.x), split30(b.y));
            a = make_ulonglong2(split30(a.x), split30(a.y));
        }
        if (KSM) {
            kpark[(d * 2 + 0) * blockDim.x + threadIdx.x] = b;
            kpark[(d * 2 + 1) * blockDim.x + threadIdx.x] = a;
        } else {
            kb[KSM ? 0 : d] = b;
            ka[KSM ? 0 : d] = a;
        }
    }
    auto KB = [&](int d) { return KSM ? kpark[(d * 2 + 0) * blockDim.x + threadIdx.x] : kb[KSM ? 0 : d]; };
    auto KA = [&](int d) { return KSM ? kpark[(d * 2 + 1) * blockDim.x + threadIdx.x] : ka[KSM ? 0 : d]; };
    for (int f = 0; f < ncol; f++) {
        ulonglong2 r0, r1;
        if (SPLIT) {
            u64 a[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int d = 0; d < BETA; d++) {
                const u64 *limb = d == own ? lane + (((size_t)f * 2 + 1) * ls + i) * N
                                           : digits + (((size_t)f * BETA + d) * E + i) * N;
                ulonglong2 v = gather_pair(limb, sx, swap);
                v = make_ulonglong2(split30(v.x), split30(v.y));
                const ulonglong2 b = KB(d), kk = KA(d);
                mac_split(a[0], a[1], a[2], v.x, b.x);
                mac_split(a[3], a[4], a[5], v.y, b.y);
                mac_split(a[6], a[7], a[8], v.x, kk.x);
                mac_split(a[9], a[10], a[11], v.y, kk.y);
            }
            u64 h[4] = {0, 0, 0, 0}, l[4] = {0, 0, 0, 0};
#pragma unroll
            for (int c = 0; c < 4; c++) fold30(h[c], l[c], a[3 * c], a[3 * c + 1], a[3 * c + 2]);
            r0 = make_ulonglong2(redc(h[0], l[0], P), redc(h[1], l[1], P));
            r1 = make_ulonglong2(redc(h[2], l[2], P), redc(h[3], l[3], P));
        } else {
            u64 h0 = 0, l0 = 0, h1 = 0, l1 = 0, h2 = 0, l2 = 0, h3 = 0, l3 = 0;
#pragma unroll
            for (int d = 0; d < BETA; d++) {
                const u64 *limb = d == own ? lane + (((size_t)f * 2 + 1) * ls + i) * N
                                           : digits + (((size_t)f * BETA + d) * E + i) * N;
                const ulonglong2 v = gather_pair(limb, sx, swap);
                const ulonglong2 b = KB(d), kk = KA(d);
                mac128(h0, l0, v.x, b.x);
                mac128(h1, l1, v.y, b.y);
                mac128(h2, l2, v.x, kk.x);
                mac128(h3, l3, v.y, kk.y);
            }
            r0 = make_ulonglong2(redc(h0, l0, P), redc(h1, l1, P));
            r1 = make_ulonglong2(redc(h2, l2, P), redc(h3, l3, P));
        }
        if (pmodq && i <= level) {
            const ulonglong2 c0 = gather_pair(lane + (((size_t)f * 2) * ls + i) * N, sx, swap);
            const u64 pw = pmodq[2 * i], pws = pmodq[2 * i + 1];
            r0.x = add_mod(r0.x, shoup_mul(c0.x, pw, pws, P.q), P.q);
            r0.y = add_mod(r0.y, shoup_mul(c0.y, pw, pws, P.q), P.q);
        }
        *reinterpret_cast<ulonglong2 *>(u + (((size_t)f * 2 + 0) * E + i) * N + x) = r0;
        *reinterpret_cast<ulonglong2 *>(u + (((size_t)f * 2 + 1) * E + i) * N + x) = r1;
    }
}

// ------------------------------------------------------------------------
// ModDown finish + masked accumulation (the SpIntra-CA products):
//   R_p = (u_p - conv_p) * P^-1  (+ phi_g(c0) for p = 0)
//   out_d += mask_d (x) R         (mask in Montgomery form; null mask: out_d = R)
// ------------------------------------------------------------------------
constexpr int kMaxDest = 8;
struct DestList {
    int n;
    int out_ls;
    u64 *out[kMaxDest];
    const u64 *mask[kMaxDest];
};

__global__ void __launch_bounds__(256)
k_moddown_finish_mac(const u64 *__restrict__ u, int E, const u64 *__restrict__ conv,
                     const u64 *__restrict__ lane, int ls, int ncol, int level, uint32_t g,
                     int log_n, const u64 *__restrict__ pinv, const DestList dl,
                     const PrimeC *__restrict__ primes)
{
    const int N = 1 << log_n;
    const int i = blockIdx.y;
    const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= N) return;
    const PrimeC P = primes[i];
    const u64 q = P.q, pv = pinv[2 * i], pvs = pinv[2 * i + 1];
    const int sx = auto_src(x, g, log_n);
    const bool swap = sx & 1;
    const int nl = level + 1;
    ulonglong2 m[kMaxDest];
#pragma unroll
    for (int d = 0; d < kMaxDest; d++)
        if (d < dl.n && dl.mask[d])
            m[d] = *reinterpret_cast<const ulonglong2 *>(dl.mask[d] + (size_t)i * N + x);
    for (int f = 0; f < ncol; f++) {
#pragma unroll
        for (int p = 0; p < 2; p++) {
            const int poly = f * 2 + p;
            const ulonglong2 uu = *reinterpret_cast<const ulonglong2 *>(u + ((size_t)poly * E + i) * N + x);
            const ulonglong2 cc = *reinterpret_cast<const ulonglong2 *>(conv + ((size_t)poly * nl + i) * N + x);
            u64 r0 = shoup_mul(sub_mod(uu.x, cc.x, q), pv, pvs, q);
            u64 r1 = shoup_mul(sub_mod(uu.y, cc.y, q), pv, pvs, q);
            if (p == 0) {
                const ulonglong2 c0 = gather_pair(lane + ((size_t)(f * 2) * ls + i) * N, sx, swap);
                r0 = add_mod(r0, c0.x, q);
                r1 = add_mod(r1, c0.y, q);
            }
#pragma unroll
            for (int d = 0; d < kMaxDest; d++) {
                if (d < dl.n) {
                    ulonglong2 *o = reinterpret_cast<ulonglong2 *>(dl.out[d] + ((size_t)poly * dl.out_ls + i) * N + x);
                    if (dl.mask[d]) {
                        ulonglong2 ov = *o;
                        ov.x = add_mod(ov.x, mont_mul(r0, m[d].x, P), q);
                        ov.y = add_mod(ov.y, mont_mul(r1, m[d].y, P), q);
                        *o = ov;
                    } else {
                        *o = make_ulonglong2(r0, r1);
                    }
                }
            }
        }
    }
}

// out_d += mask_d (x) lane (the kept values of a lane, rotation 0)
__global__ void __launch_bounds__(256)
k_stay_mac(const u64 *__restrict__ lane, int ls, int ncol, int level, const DestList dl,
           const PrimeC *__restrict__ primes, int N)
{
    const int i = blockIdx.y;
    const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= N) return;
    const PrimeC P = primes[i];
    ulonglong2 m[kMaxDest];
#pragma unroll
    for (int d = 0; d < kMaxDest; d++)
        if (d < dl.n) m[d] = *reinterpret_cast<const ulonglong2 *>(dl.mask[d] + (size_t)i * N + x);
    for (int f = 0; f < ncol; f++) {
#pragma unroll
        for (int p = 0; p < 2; p++) {
            const int poly = f * 2 + p;
            const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(lane + ((size_t)poly * ls + i) * N + x);
#pragma unroll
            for (int d = 0; d < kMaxDest; d++) {
                if (d < dl.n) {
                    ulonglong2 *o = reinterpret_cast<ulonglong2 *>(dl.out[d] + ((size_t)poly * dl.out_ls + i) * N + x);
                    ulonglong2 ov = *o;
                    ov.x = add_mod(ov.x, mont_mul(v.x, m[d].x, P), P.q);
                    ov.y = add_mod(ov.y, mont_mul(v.y, m[d].y, P), P.q);
                    *o = ov;
                }
            }
        }
    }
}

// ------------------------------------------------------------------------
// One SpIntra-CA group, all outputs at once (double hoisting): for each
// output d,  ext_d = sum over its rotated sources r of mask (x) (u_r +
// P phi_r(c0)) + sum over its kept sources of mask (x) P lane, in the
// extended basis q_0..q_l, p_0..p_{K-1} (the P terms vanish mod p_k).
// ModDown(ext_d) is then exactly the sum of mask (x) Rot and mask (x) lane,
// since ModDown(A + P B) = ModDown(A) + B.
// ------------------------------------------------------------------------

// Partial sums are products v * m~ (m~ = mask R mod q, its Montgomery form)
// added without reduction; one Montgomery reduction of the total gives
// sum v * m mod q.  That needs total < q 2^64: every product is below
// q^2 < 2^120, so up to 255 terms per output and launch are safe after
// folding the high word mod q (a launch takes at most kGmacSrc sources, and
// each source feeds an output at most once).
//
// For primes below 2^46 both factors are split into 23-bit halves,
// v = v0 + v1 2^23, and the three partial sums  A0 = sum v0 m0,
// A1 = sum (v0 m1 + v1 m0), A2 = sum v1 m1  are kept in 64-bit words
// (below 2^55 for 255 terms): four 32 x 32 -> 64-bit multiply-adds per
// product instead of a 64 x 64 -> 128-bit one.  The halves are stored as
// v0 | v1 << 32, so each factor is a register pair read without shifts.
// Other primes (q_0 and the special primes, up to 60 bits) are split into
// 30-bit halves and folded into a 128-bit sum every 8 terms.
//
// Tiling.  A tile is PPC polynomials (column, part) times PPN neighbouring
// slot pairs of one limb, thread = one polynomial at one slot pair (PPC =
// min(npoly, 16), PPN = min(128 / PPC, 16): for 32 polynomials two tiles of
// 16 x 8, 128-byte runs per polynomial).  A CTA holds one tile and G thread
// groups that share its staged words: every group copies and splits a share
// of the sources and masks, then computes its own contiguous slice of the
// outputs (balanced by term count on the host).  With seven or more outputs
// G = 3: the CTA gets three times the warps for the same shared memory
// (measured on a 66-source, 12-output group: 9% faster than one group);
// with fewer, the per-thread setup of extra groups costs more than it
// hides (6 outputs: one group 20% faster than three), so G = 1.  Phase 1
// copies the sources (the key-switch output, which already holds u +
// P phi(c0), or the kept lane) and the tile's mask words into shared memory
// with asynchronous copies, all in flight at once; phase 2 turns kept lanes
// into P lane and splits words in place; phase 3 walks the group's
// outputs, each a register sum over its terms.
constexpr int kGmacTile = 128;    // threads per group: PPC x PPN (idle ones when npoly < 8)
constexpr int kGmacGroups = 3;    // most output groups per CTA
constexpr int kGmacThreads = kGmacTile * kGmacGroups;
constexpr int kGmacOut = 64;      // outputs per launch

// the launch's program, passed by value (kernel parameters sit in the
// constant bank: uniform reads need no global loads)
struct GProg {
    int nsrc, nterm, X, accumulate;
    int ppc, ppn;                       // tile: polynomials x slot pairs
    int groups;                         // thread groups (blockDim = groups x kGmacTile)
    int gfirst[kGmacGroups + 1];        // first output of each thread group
    const u64 *su[kern::kGmacSrc];      // rotation: key-switch output; kept lane: nullptr
    const u64 *slane[kern::kGmacSrc];   // kept lane
    u32 tvoff[kern::kGmacTerms];        // terms sorted by output: byte offset of the source's row in vsm
    const u64 *tmask[kern::kGmacTerms];
    int dfirst[kGmacOut + 1];
    u64 *outs[kGmacOut];
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// 16-byte shared-memory load by 32-bit shared address (volatile: it must
// stay after the barrier that publishes the staged words)
__device__ __forceinline__ ulonglong2 lds128(u32 addr)
{
    ulonglong2 v;
    asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "r"(addr));
    return v;
}

// MINB: CTAs of kGmacThreads threads per SM the registers are budgeted for
// (2: up to 85 registers a thread; 3: up to 56, more warps resident).
// KARA: the 23-bit split products in Karatsuba's form (mac_kara: three
// products instead of four; the same sums).
template <int MINB, bool KARA>
__global__ void __launch_bounds__(kGmacThreads, MINB)
k_group_mac(const GProg pg, int ncol, int level, int E, int ls, int log_n,
            const u64 *__restrict__ pmodq, const PrimeC *__restrict__ primes, int nq)
{
    extern __shared__ __align__(16) unsigned char gsm[];
    const int npoly = 2 * ncol, PPC = pg.ppc, PPN = pg.ppn;
    const int npg = (npoly + PPC - 1) / PPC;
    const int nsrc = pg.nsrc, nterm = pg.nterm;
    ulonglong2 *vsm = reinterpret_cast<ulonglong2 *>(gsm);                  // [nsrc][kGmacTile]
    ulonglong2 *msm = vsm + (size_t)nsrc * kGmacTile;                       // [nterm][PPN]
    const int N = 1 << log_n;
    const int grp = threadIdx.x / kGmacTile, lt = threadIdx.x % kGmacTile;
    const int pl = lt / PPN, pp = lt - pl * PPN;
    const int pgi = blockIdx.x % npg, blk = blockIdx.x / npg;
    const int poly = pgi * PPC + pl;
    const int x = 2 * (blk * PPN + pp);
    const bool xin = pl < PPC && x < N;          // a slot pair of the tile
    const bool act = xin && poly < npoly;        // ... of an existing polynomial
    const int i = blockIdx.y;
    const bool isq = i <= level;
    const PrimeC P = primes[isq ? i : nq + (i - level - 1)];
    const u64 q = P.q;
    const bool split = q < (1ull << 46);
    const size_t ext_off = ((size_t)poly * E + i) * N + x;
    const int G = pg.groups;
    // 1. asynchronous copies: the masks of terms grp PPC + pl (step G PPC)
    // at this slot pair, the sources grp, grp + G, ... of this thread's slot
    if (xin)
        for (int t = grp * PPC + pl; t < nterm; t += G * PPC)
            cp_async16(msm + t * PPN + pp, pg.tmask[t] + (size_t)i * N + x);
    if (act) {
        for (int s = grp; s < nsrc; s += G) {
            ulonglong2 *dst = vsm + (size_t)s * kGmacTile + lt;
            if (pg.su[s]) cp_async16(dst, pg.su[s] + ext_off);
            else if (isq) cp_async16(dst, pg.slane[s] + ((size_t)poly * ls + i) * N + x);
            else *dst = make_ulonglong2(0, 0);   // P lane vanishes mod the special primes
        }
    }
    cp_async_wait_all();
    // 2. in place, each thread on the words it copied: kept lanes times P,
    // every word split into halves (23 bits below 2^46, else 30 bits)
    if (xin)
        for (int t = grp * PPC + pl; t < nterm; t += G * PPC) {
            const ulonglong2 m = msm[t * PPN + pp];
            msm[t * PPN + pp] = split ? make_ulonglong2(split23(m.x), split23(m.y))
                                      : make_ulonglong2(split30(m.x), split30(m.y));
        }
    if (act) {
        const u64 pw = isq ? pmodq[2 * i] : 0, pws = isq ? pmodq[2 * i + 1] : 0;
        for (int s = grp; s < nsrc; s += G) {
            const bool kept = isq && !pg.su[s];
            ulonglong2 *dst = vsm + (size_t)s * kGmacTile + lt;
            ulonglong2 v = *dst;
            if (kept) {
                v.x = shoup_mul(v.x, pw, pws, q);
                v.y = shoup_mul(v.y, pw, pws, q);
            }
            *dst = split ? make_ulonglong2(split23(v.x), split23(v.y))
                         : make_ulonglong2(split30(v.x), split30(v.y));
        }
    }
    __syncthreads();
    if (!act) return;
    // 3. this group's outputs.  Shared-memory reads by 32-bit address: the
    // source row of a term is a constant offset from this thread's slot, the
    // mask row steps by PPN words per term.
    const int d0 = pg.gfirst[grp], d1 = pg.gfirst[grp + 1];
    const u32 vbase = (u32)__cvta_generic_to_shared(vsm + lt);
    const u32 mstep = (u32)PPN * 16;
    u32 maddr = (u32)__cvta_generic_to_shared(msm + pp) + (u32)pg.dfirst[d0] * mstep;
    for (int d = d0; d < d1; d++) {
        ulonglong2 *o = reinterpret_cast<ulonglong2 *>(pg.outs[d] + ext_off);
        const ulonglong2 b = pg.accumulate ? *o : make_ulonglong2(0, 0);
        const int t0 = pg.dfirst[d], t1 = pg.dfirst[d + 1];
        ulonglong2 r;
        if (split) {
            u64 a0 = 0, a1 = 0, a2 = 0, c0 = 0, c1 = 0, c2 = 0;
            if (KARA) {
                for (int t = t0; t < t1; t++, maddr += mstep) {
                    const ulonglong2 v = lds128(vbase + pg.tvoff[t]);
                    const ulonglong2 m = lds128(maddr);
                    mac_kara(a0, a1, a2, v.x, m.x);
                    mac_kara(c0, c1, c2, v.y, m.y);
                }
                r = make_ulonglong2(fold_kara(a0, a1, a2, P), fold_kara(c0, c1, c2, P));
            } else {
                for (int t = t0; t < t1; t++, maddr += mstep) {
                    const ulonglong2 v = lds128(vbase + pg.tvoff[t]);
                    const ulonglong2 m = lds128(maddr);
                    mac_split(a0, a1, a2, v.x, m.x);
                    mac_split(c0, c1, c2, v.y, m.y);
                }
                r = make_ulonglong2(fold_split(a0, a1, a2, P), fold_split(c0, c1, c2, P));
            }
        } else {
            // 30-bit halves: partial sums folded into 128 bits every 8 terms
            u64 lo0 = 0, hi0 = 0, lo1 = 0, hi1 = 0;
            for (int t = t0; t < t1;) {
                const int te = min(t + 8, t1);
                u64 a0 = 0, a1 = 0, a2 = 0, c0 = 0, c1 = 0, c2 = 0;
                for (; t < te; t++, maddr += mstep) {
                    const ulonglong2 v = lds128(vbase + pg.tvoff[t]);
                    const ulonglong2 m = lds128(maddr);
                    mac_split(a0, a1, a2, v.x, m.x);
                    mac_split(c0, c1, c2, v.y, m.y);
                }
                fold30(hi0, lo0, a0, a1, a2);
                fold30(hi1, lo1, c0, c1, c2);
            }
            r = make_ulonglong2(redc(reduce_word(hi0, P), lo0, P), redc(reduce_word(hi1, P), lo1, P));
        }
        if (pg.accumulate) {
            r.x = add_mod(r.x, b.x, q);
            r.y = add_mod(r.y, b.y, q);
        }
        *o = r;
    }
}

// ModDown followed by the rescale by q_l, equal word for word to the two
// done in turn.  With conv_i the base conversion of the special limbs and
// o_l = (ext_l - conv_l) P^-1 mod q_l (coefficient domain: the limb the
// rescale drops), the rescaled limbs are
//   ((ext_i - conv_i) P^-1 - [o_l]_{q_i}) q_l^-1 = (ext_i - (conv_i + P o_l)) (P q_l)^-1,
// so one forward NTT of w_i = conv_i + P o_l mod q_i per kept limb replaces
// the NTT of conv_i and the rescale's NTT of [o_l]_{q_i}.  The conversion
// is centred (see k_moddown_conv) and the rescale rounds: its offset
// (q_l - 1) / 2, seen before the division by P, is H = P (q_l - 1) / 2,
// which vanishes on the special limbs, enters limb l through o_l and the
// kept limbs as w_i - [H]_{q_i}.
// ext: [npoly][E][N], limbs l and l+1.. in the coefficient domain;
// w: [npoly][l][N] coefficient domain.
template <int NMAX>
__global__ void __launch_bounds__(256)
k_moddown_rescale_conv(const u64 *__restrict__ ext, int E, u64 *w, int l,
                       const ConvTab *__restrict__ tab, const u64 *__restrict__ pinv,
                       const u64 *__restrict__ pmodq, const u64 *__restrict__ hq,
                       const PrimeC *__restrict__ primes, int N)
{
    const int poly = blockIdx.y;
    const ConvTab &T = *tab;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    u64 y[NMAX];
    const int c = conv_inputs<NMAX>(T, ext + (size_t)poly * E * N + x, N, y, primes);
    const PrimeC Pl = primes[l];
    // hq[i] = [H]_{q_i}, H = P (q_l - 1) / 2
    const u64 el = add_mod(ext[((size_t)poly * E + l) * N + x], hq[l], Pl.q);
    const u64 ol = shoup_mul(sub_mod(el, conv_point<NMAX>(T, y, l, Pl, c), Pl.q), pinv[2 * l],
                             pinv[2 * l + 1], Pl.q);
    for (int t = 0; t < l; t++) {
        const PrimeC P = primes[t];
        w[((size_t)poly * l + t) * N + x] =
            sub_mod(add_mod(conv_point<NMAX>(T, y, t, P, c), shoup_mul(ol, pmodq[2 * t], pmodq[2 * t + 1], P.q),
                            P.q), hq[t], P.q);
    }
}

// out_i = (ext_i - w_i) (P q_l)^-1 for i < l (NTT domain)
__global__ void __launch_bounds__(256)
k_moddown_rescale_finish(const u64 *__restrict__ ext, int E, const u64 *__restrict__ w, u64 *out,
                         int ls, int npoly, int l, const u64 *__restrict__ tab,
                         const PrimeC *__restrict__ primes, int N)
{
    const int i = blockIdx.y;
    const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= N) return;
    const u64 q = primes[i].q, c = tab[2 * i], cs = tab[2 * i + 1];
    for (int poly = 0; poly < npoly; poly++) {
        const ulonglong2 e = *reinterpret_cast<const ulonglong2 *>(ext + ((size_t)poly * E + i) * N + x);
        const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(w + ((size_t)poly * l + i) * N + x);
        *reinterpret_cast<ulonglong2 *>(out + ((size_t)poly * ls + i) * N + x) =
            make_ulonglong2(shoup_mul(sub_mod(e.x, v.x, q), c, cs, q),
                            shoup_mul(sub_mod(e.y, v.y, q), c, cs, q));
    }
}

// ModDown + rescale at N = 2^16, the conversion fused into the first NTT
// pass of w (see k_moddown_rescale_conv for what w is).  First
// k_moddown_prep, per coefficient of each polynomial: y_k (the inverse NTT
// of the special limbs scaled to [u_k (P/p_k)^-1]_{p_k}), c = #{y_k > p_k/2},
// o_l = ((ext_l + [H]_{q_l}) - Conv_l(y) + c [P]_{q_l}) P^-1 mod q_l, and
// o_l | c << 60 written over limb l (q_l < 2^60; limb l is not read again).
// Then k_moddown_ntt16_a per (column tile, kept limb t, polynomial): w_t =
// Conv_t(y, c) + P o_l - [H]_{q_t} mod q_t, straight into pass A of w_t.
template <int NMAX>
__global__ void __launch_bounds__(256)
k_moddown_prep(u64 *ext, int E, int l, const ConvTab *__restrict__ tab, const u64 *__restrict__ pinv,
               const u64 *__restrict__ hq, const PrimeC *__restrict__ primes, int N)
{
    const int poly = blockIdx.y;
    const ConvTab &T = *tab;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    u64 y[NMAX];
    int c = 0;
    const u64 *src = ext + (size_t)poly * E * N + x;
#pragma unroll
    for (int k = 0; k < NMAX; k++)
        if (k < T.n_in) {
            const u64 yk = src[(size_t)T.in_l[k] * N];
            c += yk > (primes[T.in_p[k]].q >> 1);
            y[k] = split30(yk);
        }
    const PrimeC Pl = primes[l];
    u64 *el = ext + ((size_t)poly * E + l) * N + x;
    const u64 e = add_mod(*el, hq[l], Pl.q);
    const u64 ol = shoup_mul(sub_mod(e, conv_point<NMAX>(T, y, l, Pl, c), Pl.q), pinv[2 * l], pinv[2 * l + 1], Pl.q);
    *el = ol | ((u64)c << 60);
}

template <int NMAX, bool OD>
__global__ void __launch_bounds__(256, OD ? 4 : 3)
k_moddown_ntt16_a(const u64 *__restrict__ ext, int E, u64 *w, int l, const ConvTab *__restrict__ tab,
                  const u64 *__restrict__ pmodq, const u64 *__restrict__ hq,
                  const PrimeC *__restrict__ primes, const ulonglong2 *__restrict__ tw)
{
    const int t = blockIdx.y, poly = blockIdx.z;
    const ConvTab &T = *tab;
    __shared__ u64 sm[256 * 16];
    __shared__ ulonglong2 stw[256];
    const PrimeC P = primes[t];
    const ulonglong2 *twp = tw + (size_t)t * 65536;
    stw[threadIdx.x] = twp[threadIdx.x];
    const u64 pw = pmodq[2 * t], pws = pmodq[2 * t + 1], ht = hq[t];
    u64 hm_[NMAX], nb = T.negb[t];
#pragma unroll
    for (int k = 0; k < NMAX; k++) hm_[k] = k < T.n_in ? T.hmod[k][t] : 0;
    const u64 *base = ext + (size_t)poly * E * 65536;
    const int c = threadIdx.x & 15, r = threadIdx.x >> 4, c0 = blockIdx.x * 16;
    u64 v[16];
#pragma unroll
    for (int m = 0; m < 16; m++) {
        const size_t idx = (size_t)(r + 16 * m) * 256 + c0 + c;
        const u64 pk = base[(size_t)l * 65536 + idx];
        const u64 ol = pk & ((1ull << 60) - 1);
        const int cc = (int)(pk >> 60);
        u64 a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
        for (int k = 0; k < NMAX; k++)
            if (k < T.n_in) mac_split(a0, a1, a2, split30(base[(size_t)T.in_l[k] * 65536 + idx]), hm_[k]);
        if (cc) mac_split(a0, a1, a2, (u64)cc, nb);
        u64 hi = 0, lo = 0;
        fold30(hi, lo, a0, a1, a2);
        const u64 conv = redc(hi, lo, P);
        v[m] = sub_mod(add_mod(conv, shoup_mul(ol, pw, pws, P.q), P.q), ht, P.q);
    }
    __syncthreads();   // stw
    u64 *d = w + ((size_t)poly * l + t) * 65536 + c0;
    if (P.q < (1ull << 47)) fwd_a16_rounds<true, 16, OD>(v, d, stw, P.q, sm);
    else fwd_a16_rounds<false, 16, OD>(v, d, stw, P.q, sm);
}

// residues mod the special primes of a polynomial given by its limb 0,
// read as a centred integer (valid when |coefficient| < q_0 / 2)
__global__ void k_lift_special(const u64 *limb0, u64 q0, u64 *out, int np, int nq,
                               const PrimeC *__restrict__ primes, int N)
{
    const int k = blockIdx.y;
    const PrimeC P = primes[nq + k];
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x) {
        const u64 v = limb0[x];
        u64 r;
        if (v <= q0 / 2) {
            r = reduce_word(v, P);
        } else {
            const u64 m = reduce_word(q0 - v, P);
            r = m ? P.q - m : 0;
        }
        out[(size_t)k * N + x] = r;
    }
}

}  // namespace

// ========================================================================
// host wrappers
// ========================================================================
// launch a kernel templated on the number of base-conversion inputs
#define FG_NIN_DISPATCH(n, LAUNCH)                                               \
    switch (n) {                                                                 \
    case 1: LAUNCH(1); break;                                                    \
    case 2: LAUNCH(2); break;                                                    \
    case 3: LAUNCH(3); break;                                                    \
    case 4: LAUNCH(4); break;                                                    \
    case 5: LAUNCH(5); break;                                                    \
    case 6: LAUNCH(6); break;                                                    \
    case 7: LAUNCH(7); break;                                                    \
    case 8: LAUNCH(8); break;                                                    \
    default: throw fg_error(FG_EINVAL, "base conversion with more than 8 inputs"); \
    }

namespace kern {

KTimer::KTimer(fg_ctx *c, const char *cls, double alg_bytes) : ctx(c), bytes(alg_bytes)
{
    g_launch_ctx = c;
    on = !c->time_class.empty() && c->time_class == cls;
    if (on) {
        a = c->event();
        cudaEventRecord(a, c->stream);
    }
}

KTimer::~KTimer()
{
    if (on) {
        cudaEvent_t b = ctx->event();
        cudaEventRecord(b, ctx->stream);
        ctx->timed.push_back({a, b, bytes});
    }
}


template <int COLS, int ROWS, bool OD>
static void ntt16_launch_t(fg_ctx *ctx, const Batch &bt, int count, bool inverse, const u64 *col_scale)
{
    const auto *fwd = (const ulonglong2 *)ctx->d_fwd;
    const auto *inv = (const ulonglong2 *)ctx->d_inv;
    dim3 gA(256 / COLS, count), gB(256 / ROWS, count);
    Batch b2 = bt;
    b2.src = b2.dst;
    b2.src_stride = b2.dst_stride;
    if (!inverse) {
        ntt16_fwd_a<COLS, OD><<<gA, 16 * COLS, 0, ctx->stream>>>(bt, ctx->d_primes, fwd);
        ntt16_fwd_b<ROWS, OD><<<gB, 16 * ROWS, 0, ctx->stream>>>(b2, ctx->d_primes, fwd,
                                                                (const ulonglong2 *)ctx->d_fwd_rows);
    } else {
        ntt16_inv_b<ROWS, OD><<<gB, 16 * ROWS, 0, ctx->stream>>>(bt, ctx->d_primes, inv,
                                                                (const ulonglong2 *)ctx->d_inv_rows);
        ntt16_inv_a<COLS, OD><<<gA, 16 * COLS, 0, ctx->stream>>>(b2, ctx->d_primes, inv, ctx->d_ninv,
                                                                col_scale);
    }
}

// the tile and twiddle form of the N = 2^16 transform from the context's tuning
template <bool OD>
static void ntt16_launch_od(fg_ctx *ctx, const Batch &bt, int count, bool inverse, const u64 *col_scale)
{
    const bool ca = ctx->tune.ntt_cols == 8, rb = ctx->tune.ntt_rows == 8;
    if (!ca && !rb) ntt16_launch_t<16, 16, OD>(ctx, bt, count, inverse, col_scale);
    else if (ca && !rb) ntt16_launch_t<8, 16, OD>(ctx, bt, count, inverse, col_scale);
    else if (!ca && rb) ntt16_launch_t<16, 8, OD>(ctx, bt, count, inverse, col_scale);
    else ntt16_launch_t<8, 8, OD>(ctx, bt, count, inverse, col_scale);
}

static void ntt16_launch(fg_ctx *ctx, const Batch &bt, int count, bool inverse,
                         const u64 *col_scale = nullptr)
{
    if (ctx->tune.ntt_tw) ntt16_launch_od<true>(ctx, bt, count, inverse, col_scale);
    else ntt16_launch_od<false>(ctx, bt, count, inverse, col_scale);
}

// N = 2^16 forward pass B alone (after a fused first pass), in place on bt.dst
template <bool OD>
static void ntt16_pass_b_od(fg_ctx *ctx, const Batch &bt, int count)
{
    const auto *fwd = (const ulonglong2 *)ctx->d_fwd;
    const auto *rows = (const ulonglong2 *)ctx->d_fwd_rows;
    if (ctx->tune.ntt_rows == 8)
        ntt16_fwd_b<8, OD><<<dim3(32, count), 128, 0, ctx->stream>>>(bt, ctx->d_primes, fwd, rows);
    else
        ntt16_fwd_b<16, OD><<<dim3(16, count), 256, 0, ctx->stream>>>(bt, ctx->d_primes, fwd, rows);
}

template <int LOGN>
static void ntt_launch_t(fg_ctx *ctx, const Batch &bt, int count, bool inverse)
{
    constexpr int S1 = LOGN / 2, N = 1 << LOGN, N1 = 1 << S1, N2 = N >> S1;
    constexpr int R = (kElemsB / N2) < N1 ? (kElemsB / N2) : N1;
    const size_t smA = (size_t)N1 * kColsA * 8 + (size_t)N1 * 16;
    const size_t smB = (size_t)R * N2 * 8;
    const auto *fwd = (const ulonglong2 *)ctx->d_fwd;
    const auto *inv = (const ulonglong2 *)ctx->d_inv;
    dim3 gA(N2 / kColsA, count), gB(N1 / R, count);
    Batch b2 = bt;
    b2.src = b2.dst;
    b2.src_stride = b2.dst_stride;
    if (!inverse) {
        ntt_fwd_a<LOGN><<<gA, kNttThreads, smA, ctx->stream>>>(bt, ctx->d_primes, fwd);
        ntt_fwd_b<LOGN><<<gB, kNttThreads, smB, ctx->stream>>>(b2, ctx->d_primes, fwd);
    } else {
        ntt_inv_b<LOGN><<<gB, kNttThreads, smB, ctx->stream>>>(bt, ctx->d_primes, inv);
        ntt_inv_a<LOGN><<<gA, kNttThreads, smA, ctx->stream>>>(b2, ctx->d_primes, inv, ctx->d_ninv);
    }
}

static void launch_ntt(fg_ctx *ctx, const LimbSet &src, const LimbSet &dst, bool inverse)
{
    FG_CHECK(src.per_row == dst.per_row && src.rows == dst.rows, FG_EINVAL, "ntt: shape mismatch");
    if (src.rows == 0 || src.per_row == 0) return;
    Batch bt = make_batch(src.base, src.stride, dst.base, dst.stride, src.per_row, src.rows,
                          src.pidx);
    const int count = src.rows * src.per_row;
    FG_CHECK(count <= 65535, FG_EINVAL, "ntt: more than 65535 limbs in one batch");
    int active = 0;
    for (int v : src.pidx) active += v >= 0;
    KTimer kt(ctx, "ntt", (double)active * src.rows * ctx->n * 8 * 2);
    switch (ctx->log_n) {
    case 10: ntt_launch_t<10>(ctx, bt, count, inverse); break;
    case 11: ntt_launch_t<11>(ctx, bt, count, inverse); break;
    case 12: ntt_launch_t<12>(ctx, bt, count, inverse); break;
    case 13: ntt_launch_t<13>(ctx, bt, count, inverse); break;
    case 14: ntt_launch_t<14>(ctx, bt, count, inverse); break;
    case 15: ntt_launch_t<15>(ctx, bt, count, inverse); break;
    case 16: ntt16_launch(ctx, bt, count, inverse); break;
    default: throw fg_error(FG_EINVAL, "ntt: unsupported ring degree");
    }
    check_launch("ntt", 2);
}

void ntt_fwd(fg_ctx *ctx, const LimbSet &src, const LimbSet &dst) { launch_ntt(ctx, src, dst, false); }
void ntt_inv(fg_ctx *ctx, const LimbSet &src, const LimbSet &dst) { launch_ntt(ctx, src, dst, true); }

static inline dim3 ew_grid(int N, int count) { return dim3((N + 255) / 256, count); }

static Batch contiguous(u64 *p, int count, const std::vector<int> &pidx)
{
    const int per = (int)pidx.size();
    return make_batch(p, per, p, per, per, count / per, pidx);
}

void to_mont(fg_ctx *ctx, u64 *data, int count, const std::vector<int> &pidx)
{
    if (!count) return;
    KTimer kt(ctx, "to_mont", 0);
    k_to_mont<<<ew_grid(ctx->n, count), 256, 0, ctx->stream>>>(contiguous(data, count, pidx),
                                                               ctx->d_primes, ctx->n);
    check_launch("to_mont");
}

void from_mont(fg_ctx *ctx, u64 *data, int count, const std::vector<int> &pidx)
{
    if (!count) return;
    KTimer kt(ctx, "from_mont", 0);
    k_from_mont<<<ew_grid(ctx->n, count), 256, 0, ctx->stream>>>(contiguous(data, count, pidx),
                                                                 ctx->d_primes, ctx->n);
    check_launch("from_mont");
}

void pointwise(fg_ctx *ctx, const u64 *a, const u64 *b, u64 *c, int count,
               const std::vector<int> &pidx)
{
    if (!count) return;
    KTimer kt(ctx, "pointwise", 0);
    k_pointwise<<<ew_grid(ctx->n, count), 256, 0, ctx->stream>>>(
        a, b, c, contiguous(c, count, pidx), ctx->d_primes, ctx->n);
    check_launch("pointwise");
}

void add(fg_ctx *ctx, const u64 *a, const u64 *b, u64 *c, int count, const std::vector<int> &pidx)
{
    if (!count) return;
    KTimer kt(ctx, "add", 0);
    k_add<<<ew_grid(ctx->n, count), 256, 0, ctx->stream>>>(a, b, c, contiguous(c, count, pidx),
                                                           ctx->d_primes, ctx->n);
    check_launch("add");
}

void neg(fg_ctx *ctx, const u64 *a, u64 *c, int count, const std::vector<int> &pidx)
{
    if (!count) return;
    KTimer kt(ctx, "neg", 0);
    k_neg<<<ew_grid(ctx->n, count), 256, 0, ctx->stream>>>(a, c, contiguous(c, count, pidx),
                                                           ctx->d_primes, ctx->n);
    check_launch("neg");
}

void scalar(fg_ctx *ctx, const u64 *a, u64 *c, int count, const std::vector<int> &pidx,
            const u64 *d_scal)
{
    if (!count) return;
    KTimer kt(ctx, "scalar", 0);
    k_scalar<<<ew_grid(ctx->n, count), 256, 0, ctx->stream>>>(
        a, c, contiguous(c, count, pidx), ctx->d_primes, d_scal, ctx->n);
    check_launch("scalar");
}

void automorphism(fg_ctx *ctx, const u64 *a, u64 *c, int nlimbs, uint32_t g)
{
    if (!nlimbs) return;
    KTimer kt(ctx, "automorphism", 0);
    k_automorphism<<<ew_grid(ctx->n, nlimbs), 256, 0, ctx->stream>>>(a, c, nlimbs, g, ctx->log_n);
    check_launch("automorphism");
}

void small_to_res(fg_ctx *ctx, const int8_t *e, u64 *out, int n_limbs, const int *d_pidx)
{
    KTimer kt(ctx, "small_to_res", 0);
    k_small_to_res<<<ew_grid(ctx->n, n_limbs), 256, 0, ctx->stream>>>(e, out, d_pidx,
                                                                      ctx->d_primes, ctx->n);
    check_launch("small_to_res");
}

void expand_uniform(fg_ctx *ctx, cudaStream_t st, u64 *ct, size_t ct_pitch, const u64 *c0, int ncols,
                    int nl, u64 seed, u64 index0)
{
    if (!ncols || !nl) return;
    FG_CHECK(ncols <= 65535 && nl <= ctx->nq, FG_EINVAL, "expand_uniform: bad shape");
    dim3 g((ctx->n + 255) / 256, nl, ncols);
    k_expand_uniform<<<g, 256, 0, st>>>(ct, ct_pitch, c0, nl, seed, hm::kSeededPurpose, index0,
                                        ctx->d_primes, ctx->n);
    check_launch("expand_uniform");
}

void copy_limbs(fg_ctx *ctx, const u64 *src, int src_ls, u64 *dst, int dst_ls, int npoly, int nl)
{
    if (!npoly || !nl) return;
    KTimer kt(ctx, "copy", (double)npoly * nl * ctx->n * 16);
    dim3 g((ctx->n + 255) / 256, nl, npoly);
    k_copy_limbs<<<g, 256, 0, ctx->stream>>>(src, src_ls, dst, dst_ls, nl, ctx->n);
    check_launch("copy_limbs");
}

void comb_const_mac(fg_ctx *ctx, const u64 *X, int F, int Fp, int level, const u64 *consts, u64 *Z,
                    int z_ls, int fb, int fe, bool accumulate)
{
    // split partial sums stay below 2^64 for up to 2^16 terms
    FG_CHECK(F < (1 << 16), FG_EINVAL, "combination over more than 2^16 input columns");
    if (fe < 0) fe = F;
    FG_CHECK(0 <= fb && fb < fe && fe <= F, FG_EINVAL, "combination column range");
    const int nj = (Fp + kCombJ - 1) / kCombJ;
    // inputs read once, outputs written once (read too when accumulating)
    KTimer kt(ctx, "comb", ((double)(fe - fb) + Fp * (accumulate ? 2 : 1)) * 2 * (level + 1) * ctx->n * 8);
    dim3 g(((ctx->n + 255) / 256) * nj, level + 1, 2);
    k_comb<<<g, 256, 0, ctx->stream>>>(X, F, fb, fe, accumulate ? 1 : 0, Fp, nj, level, consts, Z, z_ls,
                                       ctx->d_primes, ctx->n);
    check_launch("comb");
}

void rescale_coef(fg_ctx *ctx, const u64 *in, int in_ls, u64 *out, int out_ls, int npoly, int level)
{
    FG_CHECK(level >= 1, FG_ELEVEL, "rescale needs level >= 1");
    KTimer kt(ctx, "rescale", (double)npoly * (2 * level + 1) * ctx->n * 8);
    dim3 g((ctx->n + 255) / 256, level, npoly);
    k_rescale_coef<<<g, 256, 0, ctx->stream>>>(in, in_ls, out, out_ls, level, ctx->d_primes,
                                               ctx->rescale_tab(level), ctx->n);
    check_launch("rescale_coef");
}

void rescale_ntt(fg_ctx *ctx, u64 *ct, int ls, int npoly, int level)
{
    FG_CHECK(level >= 1, FG_ELEVEL, "rescale needs level >= 1");
    const int N = ctx->n;
    // top limb back to the coefficient domain (in place; it is dropped anyway)
    std::vector<int> top(ls, -1);
    top[level] = level;
    LimbSet s{ct, ls, ls, npoly, top};
    ntt_inv(ctx, s, s);
    u64 *rr = (u64 *)ctx->buf("rescale_r", (size_t)npoly * level * N * 8);
    dim3 g((N + 255) / 256, level, npoly);
    {
        KTimer kt(ctx, "rescale", (double)npoly * (level + 1) * N * 8);
        k_bcast_reduce<<<g, 256, 0, ctx->stream>>>(ct, ls, level, rr, level, ctx->d_primes, N);
        check_launch("bcast_reduce");
    }
    std::vector<int> pid(level);
    for (int i = 0; i < level; i++) pid[i] = i;
    LimbSet r{rr, level, level, npoly, pid};
    ntt_fwd(ctx, r, r);
    KTimer kt(ctx, "rescale", (double)npoly * level * N * 8 * 3);
    k_rescale_finish<<<g, 256, 0, ctx->stream>>>(ct, ls, rr, level, ctx->d_primes,
                                                 ctx->rescale_tab(level), N);
    check_launch("rescale_finish");
}

// ModUp at N = 2^16 with the conversion fused into the digits' first NTT
// pass: the inverse NTT of c1 scaled to give the conversion's inputs y_i,
// one kernel per (column, digit, output limb, column tile) converting and
// running stages 0..7, then pass B over every digit limb
template <bool OD>
static void modup16_fused(fg_ctx *ctx, const u64 *lane, int ls, int ncol, int level, u64 *digits)
{
    const int N = ctx->n, nl = level + 1, E = ctx->ext(level), beta = ctx->n_digits(level);
    u64 *y = (u64 *)ctx->buf("modup_c1", (size_t)ncol * nl * N * 8);
    std::vector<int> pid(nl);
    for (int i = 0; i < nl; i++) pid[i] = i;
    {
        Batch bt = make_batch(const_cast<u64 *>(lane) + (size_t)ls * N, 2 * ls, y, nl, nl, ncol, pid);
        KTimer kt(ctx, "ntt", (double)nl * ncol * N * 8 * 2);
        ntt16_launch(ctx, bt, ncol * nl, true, ctx->modup_scale_tab(level));
        check_launch("ntt", 2);
    }
    const int nmax = std::min(ctx->alpha, nl);
    int n_out = 0;
    for (int d = 0; d < beta; d++) n_out = std::max(n_out, E - std::min(ctx->alpha, nl - d * ctx->alpha));
    const ConvTab *tabs = ctx->modup_tabs(level);
    const auto *fwd = (const ulonglong2 *)ctx->d_fwd;
    {
        KTimer kt(ctx, "modup_conv", (double)ncol * (nl + (double)beta * (E - ctx->alpha)) * N * 8);
        const bool c8 = ctx->tune.ntt_cols == 8;
        dim3 g(c8 ? 32 : 16, n_out, ncol * beta);
#define FG_LAUNCH(M)                                                                                  \
        if (c8)                                                                                       \
            k_modup_ntt16_a<M, 8, OD><<<g, 128, 0, ctx->stream>>>(y, nl, digits, beta, E, tabs,       \
                                                                  ctx->d_primes, fwd);                \
        else                                                                                          \
            k_modup_ntt16_a<M, 16, OD><<<g, 256, 0, ctx->stream>>>(y, nl, digits, beta, E, tabs,      \
                                                                   ctx->d_primes, fwd)
        FG_NIN_DISPATCH(nmax, FG_LAUNCH)
#undef FG_LAUNCH
        check_launch("modup_ntt16_a");
    }
    std::vector<int> dp(beta * E);
    for (int d = 0; d < beta; d++)
        for (int i = 0; i < E; i++)
            dp[d * E + i] = (i <= level && i / ctx->alpha == d) ? -1 : ctx->ext_prime(level, i);
    Batch bd = make_batch(digits, beta * E, digits, beta * E, beta * E, ncol, dp);
    int active = 0;
    for (int v : dp) active += v >= 0;
    KTimer kt(ctx, "ntt", (double)active * ncol * N * 8 * 2 / 2);
    ntt16_pass_b_od<OD>(ctx, bd, ncol * beta * E);
    check_launch("ntt16_fwd_b");
}

void modup(fg_ctx *ctx, const u64 *lane, int ls, int ncol, int level, u64 *digits)
{
    if (ctx->log_n == 16 && ctx->tune.modup_fused) {
        if (ctx->tune.ntt_tw) modup16_fused<true>(ctx, lane, ls, ncol, level, digits);
        else modup16_fused<false>(ctx, lane, ls, ncol, level, digits);
        return;
    }
    const int N = ctx->n, nl = level + 1, E = ctx->ext(level), beta = ctx->n_digits(level);
    u64 *c1c = (u64 *)ctx->buf("modup_c1", (size_t)ncol * nl * N * 8);
    std::vector<int> pid(nl);
    for (int i = 0; i < nl; i++) pid[i] = i;
    LimbSet src{const_cast<u64 *>(lane) + (size_t)ls * N, 2 * ls, nl, ncol, pid};
    LimbSet dst{c1c, nl, nl, ncol, pid};
    ntt_inv(ctx, src, dst);
    dim3 g((N + 255) / 256, 1, ncol * beta);
    {
    KTimer kt(ctx, "modup_conv", (double)ncol * (nl + (double)beta * E - nl) * N * 8);
#define FG_LAUNCH(M)                                                                       \
    k_modup_conv<M><<<g, 256, 0, ctx->stream>>>(c1c, nl, digits, beta, E, ctx->modup_tabs(level), \
                                                ctx->d_primes, N)
    FG_NIN_DISPATCH(std::min(ctx->alpha, nl), FG_LAUNCH)
#undef FG_LAUNCH
    check_launch("modup_conv");
    }
    std::vector<int> dp(beta * E);
    for (int d = 0; d < beta; d++)
        for (int i = 0; i < E; i++)
            dp[d * E + i] = (i <= level && i / ctx->alpha == d) ? -1 : ctx->ext_prime(level, i);
    LimbSet ds{digits, beta * E, beta * E, ncol, dp};
    ntt_fwd(ctx, ds, ds);
}

// key-switch inner products of up to kKsMulti rotations of one lane (with
// P phi(c0) folded in when add_c0 is set)
static void ks_launch(fg_ctx *ctx, const std::vector<const KeyDev *> &keys, const std::vector<u64 *> &us,
                      const u64 *lane, int ls, int ncol, int level, const u64 *digits, bool add_c0)
{
    const int N = ctx->n, E = ctx->ext(level), beta = ctx->n_digits(level);
    FG_CHECK(beta <= kMaxBeta, FG_EINVAL, "too many key-switching digits");
    FG_CHECK(!keys.empty() && keys.size() <= (size_t)kKsMulti && keys.size() == us.size(), FG_EINVAL,
             "ks_launch: 1 to 24 rotations");
    const int KL = ctx->nq + ctx->np;
    KsSet ks;
    memset(&ks, 0, sizeof(ks));
    ks.n = (int)keys.size();
    for (int r = 0; r < ks.n; r++) {
        ks.key[r] = keys[r]->d;
        ks.g[r] = keys[r]->galois;
        ks.u[r] = us[r];
    }
    const u64 *pmodq = add_c0 ? ctx->d_pmodq : nullptr;
    dim3 g1((N / 2 + 255) / 256, ks.n, E);
    // digits and c0 once per launch, keys and outputs once per rotation
    KTimer kt(ctx, "ks_ip", ((double)ncol * beta * E + (add_c0 ? (double)ncol * (level + 1) : 0) +
                             (double)ks.n * (2.0 * beta * E + 2.0 * ncol * E)) * N * 8);
#define FG_KS_CASE(B)                                                                          \
    case B:                                                                                    \
        if (ksm && B <= 6)                                                                     \
            k_ks_ip<B, 0, (B <= 6)><<<g1, 256, (size_t)B * 2 * 256 * 16, ctx->stream>>>(         \
                ks, KL, lane, ls, digits, ncol, level, E, ctx->alpha, ctx->nq, ctx->log_n,     \
                ctx->d_primes, pmodq);                                                         \
        else if (less)                                                                         \
            k_ks_ip<B, (B <= 8 ? 1 : 0), false><<<g1, 256, 0, ctx->stream>>>(                   \
                ks, KL, lane, ls, digits, ncol, level, E, ctx->alpha, ctx->nq, ctx->log_n,     \
                ctx->d_primes, pmodq);                                                         \
        else                                                                                   \
            k_ks_ip<B, 0, false><<<g1, 256, 0, ctx->stream>>>(ks, KL, lane, ls, digits, ncol,   \
                                                              level, E, ctx->alpha, ctx->nq,   \
                                                              ctx->log_n, ctx->d_primes, pmodq); \
        break;
    const bool less = ctx->tune.ks_split == 1, ksm = ctx->tune.ks_split == 2;
    switch (beta) {
        FG_KS_CASE(1) FG_KS_CASE(2) FG_KS_CASE(3) FG_KS_CASE(4) FG_KS_CASE(5) FG_KS_CASE(6)
        FG_KS_CASE(7) FG_KS_CASE(8) FG_KS_CASE(9) FG_KS_CASE(10) FG_KS_CASE(11) FG_KS_CASE(12)
        FG_KS_CASE(13) FG_KS_CASE(14) FG_KS_CASE(15) FG_KS_CASE(16)
    default: throw fg_error(FG_EINVAL, "too many key-switching digits");
    }
#undef FG_KS_CASE
    check_launch("ks_ip");
}

void rotate_mac(fg_ctx *ctx, const KeyDev &key, const u64 *lane, int ls, int ncol, int level,
                const u64 *digits, const std::vector<Dest> &dests, int out_ls)
{
    const int N = ctx->n, nl = level + 1, E = ctx->ext(level), beta = ctx->n_digits(level);
    FG_CHECK(beta <= kMaxBeta, FG_EINVAL, "too many key-switching digits");
    const int KL = ctx->nq + ctx->np;
    u64 *u = (u64 *)ctx->buf("ks_u", (size_t)ncol * 2 * E * N * 8);
    ks_launch(ctx, {&key}, {u}, lane, ls, ncol, level, digits, false);
    std::vector<int> pp(E);
    for (int i = 0; i < E; i++) pp[i] = i <= level ? -1 : ctx->ext_prime(level, i);
    LimbSet us{u, E, E, 2 * ncol, pp};
    ntt_inv(ctx, us, us);
    u64 *conv = (u64 *)ctx->buf("ks_conv", (size_t)ncol * 2 * nl * N * 8);
    dim3 g2((N + 255) / 256, 2 * ncol);
    {
    KTimer kt(ctx, "moddown_conv", (double)2 * ncol * (ctx->np + nl) * N * 8);
#define FG_LAUNCH(M)                                                                       \
    k_moddown_conv<M><<<g2, 256, 0, ctx->stream>>>(u, E, conv, nl, ctx->moddown_tab(level),   \
                                                   ctx->d_primes, N)
    FG_NIN_DISPATCH(ctx->np, FG_LAUNCH)
#undef FG_LAUNCH
    check_launch("moddown_conv");
    }
    std::vector<int> pq(nl);
    for (int i = 0; i < nl; i++) pq[i] = i;
    LimbSet cs{conv, nl, nl, 2 * ncol, pq};
    ntt_fwd(ctx, cs, cs);
    for (size_t d0 = 0; d0 < dests.size() || d0 == 0; d0 += kMaxDest) {
        DestList dl;
        dl.n = (int)std::min<size_t>(kMaxDest, dests.size() - d0);
        dl.out_ls = out_ls;
        for (int d = 0; d < dl.n; d++) {
            dl.out[d] = dests[d0 + d].out;
            dl.mask[d] = dests[d0 + d].mask;
        }
        dim3 g3((N / 2 + 255) / 256, nl);
        int masked = 0;
        for (int d = 0; d < dl.n; d++) masked += dl.mask[d] != nullptr;
        KTimer kt(ctx, "moddown_mac",
                  ((double)5 * ncol * nl + (double)masked * nl +
                   (double)masked * ncol * 2 * nl * 2 + (double)(dl.n - masked) * ncol * 2 * nl) * N * 8);
        k_moddown_finish_mac<<<g3, 256, 0, ctx->stream>>>(u, E, conv, lane, ls, ncol, level,
                                                          key.galois, ctx->log_n,
                                                          ctx->pinv_tab(level), dl, ctx->d_primes);
        check_launch("moddown_finish_mac");
        if (dests.empty()) break;
    }
}

void stay_mac(fg_ctx *ctx, const u64 *lane, int ls, int ncol, int level,
              const std::vector<Dest> &dests, int out_ls)
{
    const int N = ctx->n;
    for (size_t d0 = 0; d0 < dests.size(); d0 += kMaxDest) {
        DestList dl;
        dl.n = (int)std::min<size_t>(kMaxDest, dests.size() - d0);
        dl.out_ls = out_ls;
        for (int d = 0; d < dl.n; d++) {
            dl.out[d] = dests[d0 + d].out;
            dl.mask[d] = dests[d0 + d].mask;
        }
        dim3 g((N / 2 + 255) / 256, level + 1);
        const int nl = level + 1;
        KTimer kt(ctx, "stay_mac", ((double)2 * ncol * nl + (double)dl.n * nl +
                                     (double)dl.n * ncol * 2 * nl * 2) * N * 8);
        k_stay_mac<<<g, 256, 0, ctx->stream>>>(lane, ls, ncol, level, dl, ctx->d_primes, N);
        check_launch("stay_mac");
    }
}


void lift_special(fg_ctx *ctx, const u64 *limb0, u64 *out)
{
    KTimer kt(ctx, "lift", 0);
    k_lift_special<<<ew_grid(ctx->n, ctx->np), 256, 0, ctx->stream>>>(limb0, ctx->primes[0], out,
                                                                      ctx->np, ctx->nq,
                                                                      ctx->d_primes, ctx->n);
    check_launch("lift_special");
}

void group_mac(fg_ctx *ctx, const std::vector<GroupSource> &srcs, const std::vector<Dest> &terms_in,
               const std::vector<int> &term_dest, const std::vector<u64 *> &outs, bool accumulate,
               int ncol, int level, int ls)
{
    const int N = ctx->n, E = ctx->ext(level), X = (int)outs.size();
    if (srcs.empty() || X == 0) return;
    FG_CHECK((int)srcs.size() <= kGmacSrc && (int)terms_in.size() <= kGmacTerms && X <= kGmacOut,
             FG_EINVAL, "group_mac: launch larger than its program limits");
    GProg pg;
    memset(&pg, 0, sizeof(pg));
    pg.nsrc = (int)srcs.size();
    pg.nterm = (int)terms_in.size();
    pg.X = X;
    pg.accumulate = accumulate ? 1 : 0;
    std::vector<int> src_of(terms_in.size());
    for (size_t s = 0; s < srcs.size(); s++) {
        pg.su[s] = srcs[s].u;
        pg.slane[s] = srcs[s].lane;
        for (int t = srcs[s].t0; t < srcs[s].t1; t++) src_of[t] = (int)s;
    }
    int n = 0;
    for (int d = 0; d < X; d++) {   // terms sorted by output
        pg.dfirst[d] = n;
        pg.outs[d] = outs[d];
        for (size_t t = 0; t < terms_in.size(); t++)
            if (term_dest[t] == d) {
                pg.tvoff[n] = (u32)src_of[t] * kGmacTile * 16;
                pg.tmask[n] = terms_in[t].mask;
                n++;
            }
    }
    pg.dfirst[X] = n;
    // thread groups and their output slices, cut where the running term
    // count passes k / G of the total
    const int G = X >= ctx->tune.gmac_groups ? kGmacGroups : 1;
    pg.groups = G;
    pg.gfirst[0] = 0;
    int k = 1;
    for (int d = 0; d < X && k < G; d++)
        while (k < G && (int64_t)pg.dfirst[d + 1] * G >= (int64_t)k * n) pg.gfirst[k++] = d + 1;
    for (; k <= kGmacGroups; k++) pg.gfirst[k] = X;
    const int npoly = 2 * ncol;
    pg.ppc = std::min(npoly, 16);
    pg.ppn = std::min(kGmacTile / pg.ppc, 16);
    const int npg = (npoly + pg.ppc - 1) / pg.ppc;
    dim3 g(((N / 2 + pg.ppn - 1) / pg.ppn) * npg, E);
    FG_CHECK(g.x < (1u << 31), FG_EINVAL, "group_mac: grid too large");
    const size_t sm = (size_t)pg.nsrc * kGmacTile * 16 + (size_t)pg.nterm * pg.ppn * 16;
    double src_limbs = 0;
    for (const auto &gs : srcs) src_limbs += gs.u ? E : level + 1;
    KTimer kt(ctx, "group_mac",
              (src_limbs * npoly + (double)pg.nterm * E +
               (double)X * npoly * E * (accumulate ? 2 : 1)) * N * 8);
    // raised once per process and size (not a stream operation, and kept out
    // of the launches a CUDA graph capture records)
    static size_t sm_set[4] = {48 * 1024, 48 * 1024, 48 * 1024, 48 * 1024};
    const int v = (ctx->tune.gmac_regs ? 1 : 0) + (ctx->tune.kara ? 2 : 0);
    auto kern = v == 0 ? k_group_mac<2, false> : v == 1 ? k_group_mac<3, false>
              : v == 2 ? k_group_mac<2, true> : k_group_mac<3, true>;
    if (sm > sm_set[v]) {
        CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        sm_set[v] = sm;
    }
    kern<<<g, G * kGmacTile, sm, ctx->stream>>>(pg, ncol, level, E, ls, ctx->log_n, ctx->d_pmodq,
                                                ctx->d_primes, ctx->nq);
    check_launch("group_mac");
}

// With ctx->tune.ks_cols = 2 the columns are split over two launches, so
// that the digits a limb's CTAs gather from L2 are half as many (the keys
// are then read once per half).
void ks_multi(fg_ctx *ctx, const std::vector<const KeyDev *> &keys, const std::vector<u64 *> &us,
              const u64 *lane, int ls, int ncol, int level, const u64 *digits)
{
    const int E = ctx->ext(level), beta = ctx->n_digits(level), N = ctx->n;
    const int parts = std::max(1, std::min(ctx->tune.ks_cols, ncol));
    for (int h = 0; h < parts; h++) {
        const int f0 = ncol * h / parts, f1 = ncol * (h + 1) / parts;
        if (f1 == f0) continue;
        for (size_t r0 = 0; r0 < keys.size(); r0 += kKsMulti) {
            const size_t r1 = std::min(keys.size(), r0 + kKsMulti);
            std::vector<u64 *> uh;
            for (size_t r = r0; r < r1; r++) uh.push_back(us[r] + (size_t)f0 * 2 * E * N);
            ks_launch(ctx, std::vector<const KeyDev *>(keys.begin() + r0, keys.begin() + r1), uh,
                      lane + (size_t)f0 * 2 * ls * N, ls, f1 - f0, level,
                      digits + (size_t)f0 * beta * E * N, true);
        }
    }
}

// ModDown + rescale at N = 2^16 with the conversion fused into w's first
// NTT pass (see k_moddown_ntt16_a)
template <bool OD>
static void moddown16_fused(fg_ctx *ctx, u64 *ext, int ncol, int level, u64 *out, int ls)
{
    const int N = ctx->n, l = level, E = ctx->ext(level), npoly = 2 * ncol;
    std::vector<int> pp(E, -1);
    pp[l] = l;
    for (int i = l + 1; i < E; i++) pp[i] = ctx->ext_prime(level, i);
    {
        Batch bt = make_batch(ext, E, ext, E, E, npoly, pp);
        KTimer kt(ctx, "ntt", (double)npoly * (ctx->np + 1) * N * 8 * 2);
        ntt16_launch(ctx, bt, npoly * E, true, ctx->moddown_scale_tab(level));
        check_launch("ntt", 2);
    }
    u64 *w = (u64 *)ctx->buf("ks_conv", (size_t)npoly * l * N * 8);
    const ConvTab *tab = ctx->moddown_tab(level);
    const u64 *hq = ctx->moddown_rescale_half_tab(level);
    {
        KTimer kt(ctx, "moddown_conv", (double)npoly * (ctx->np + 2 + l) * N * 8);
        dim3 g1((N + 255) / 256, npoly);
#define FG_LAUNCH(M) \
        k_moddown_prep<M><<<g1, 256, 0, ctx->stream>>>(ext, E, l, tab, ctx->pinv_tab(level), hq, ctx->d_primes, N)
        FG_NIN_DISPATCH(ctx->np, FG_LAUNCH)
#undef FG_LAUNCH
        check_launch("moddown_prep");
        dim3 g2(16, l, npoly);
#define FG_LAUNCH(M)                                                                                \
        k_moddown_ntt16_a<M, OD><<<g2, 256, 0, ctx->stream>>>(ext, E, w, l, tab, ctx->d_pmodq, hq,    \
                                                              ctx->d_primes,                          \
                                                              (const ulonglong2 *)ctx->d_fwd)
        FG_NIN_DISPATCH(ctx->np, FG_LAUNCH)
#undef FG_LAUNCH
        check_launch("moddown_ntt16_a");
    }
    {
        std::vector<int> pq(l);
        for (int i = 0; i < l; i++) pq[i] = i;
        Batch bw = make_batch(w, l, w, l, l, npoly, pq);
        KTimer kt(ctx, "ntt", (double)npoly * l * N * 8 * 2 / 2);
        ntt16_pass_b_od<OD>(ctx, bw, npoly * l);
        check_launch("ntt16_fwd_b");
    }
    KTimer kt(ctx, "moddown_store", (double)npoly * l * 3 * N * 8);
    dim3 g3((N / 2 + 255) / 256, l);
    k_moddown_rescale_finish<<<g3, 256, 0, ctx->stream>>>(ext, E, w, out, ls, npoly, l,
                                                          ctx->moddown_rescale_tab(level), ctx->d_primes, N);
    check_launch("moddown_rescale_finish");
}

void moddown_rescale_to_lane(fg_ctx *ctx, u64 *ext, int ncol, int level, u64 *out, int ls)
{
    if (ctx->log_n == 16 && ctx->tune.moddown_fused && level >= 1) {
        if (ctx->tune.ntt_tw) moddown16_fused<true>(ctx, ext, ncol, level, out, ls);
        else moddown16_fused<false>(ctx, ext, ncol, level, out, ls);
        return;
    }
    FG_CHECK(level >= 1, FG_ELEVEL, "rescale needs level >= 1");
    const int N = ctx->n, l = level, E = ctx->ext(level), npoly = 2 * ncol;
    std::vector<int> pp(E, -1);
    pp[l] = l;
    for (int i = l + 1; i < E; i++) pp[i] = ctx->ext_prime(level, i);
    LimbSet us{ext, E, E, npoly, pp};
    ntt_inv(ctx, us, us);
    u64 *w = (u64 *)ctx->buf("ks_conv", (size_t)npoly * l * N * 8);
    {
        KTimer kt(ctx, "moddown_conv", (double)npoly * (ctx->np + 1 + l) * N * 8);
        dim3 g2((N + 255) / 256, npoly);
#define FG_LAUNCH(M)                                                                        \
        k_moddown_rescale_conv<M><<<g2, 256, 0, ctx->stream>>>(ext, E, w, l, ctx->moddown_tab(level), \
                                                               ctx->pinv_tab(level), ctx->d_pmodq,  \
                                                               ctx->moddown_rescale_half_tab(level), \
                                                               ctx->d_primes, N)
        FG_NIN_DISPATCH(ctx->np, FG_LAUNCH)
#undef FG_LAUNCH
        check_launch("moddown_rescale_conv");
    }
    std::vector<int> pq(l);
    for (int i = 0; i < l; i++) pq[i] = i;
    LimbSet ws{w, l, l, npoly, pq};
    ntt_fwd(ctx, ws, ws);
    KTimer kt(ctx, "moddown_store", (double)npoly * l * 3 * N * 8);
    dim3 g3((N / 2 + 255) / 256, l);
    k_moddown_rescale_finish<<<g3, 256, 0, ctx->stream>>>(ext, E, w, out, ls, npoly, l,
                                                          ctx->moddown_rescale_tab(level),
                                                          ctx->d_primes, N);
    check_launch("moddown_rescale_finish");
}

}  // namespace kern
