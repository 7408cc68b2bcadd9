// fg_internal.h -- host-side structures shared by the library's translation
// units (context, keys, plan) and the kernel launch wrappers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/ficgcn.h"

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;

// ------------------------------------------------------------------ errors
// Internal code throws fg_error; every C entry point catches it and turns it
// into a status code plus fg_last_error text.
struct fg_error : std::runtime_error {
    int code;
    fg_error(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

#define FG_CHECK(cond, code, msg)                                   \
    do {                                                            \
        if (!(cond)) throw fg_error((code), (msg));                 \
    } while (0)

#define CUDA_TRY(call)                                                              \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess)                                                      \
            throw fg_error(e_ == cudaErrorMemoryAllocation ? FG_EOOM : FG_ECUDA,    \
                           std::string(#call) + ": " + cudaGetErrorString(e_));    \
    } while (0)

// ------------------------------------------------------------------ host math
namespace hm {
u64 mulmod(u64 a, u64 b, u64 q);
u64 powmod(u64 a, u64 e, u64 q);
u64 invmod(u64 a, u64 q);
bool is_prime(u64 n);
std::vector<u64> gen_primes(int log_n, const std::vector<int> &bits);
u64 find_psi(int n, u64 q);
u64 shoup(u64 w, u64 q);          // floor(w 2^64 / q)
u64 mont_qneg(u64 q);             // -q^-1 mod 2^64
u64 to_mont(u64 x, u64 q);        // x 2^64 mod q
int bitrev(int x, int bits);

// SplitMix64 streams (see ficgcn.h)
struct Stream {
    u64 s;
    Stream(u64 seed, u64 purpose, u64 index);
    u64 next();
};
void sample_ternary(u64 seed, u64 purpose, u64 index, int n, int8_t *out);
void sample_gauss(u64 seed, u64 purpose, u64 index, int n, int8_t *out);
void sample_uniform(u64 seed, u64 purpose, u64 index, const u64 *primes, int n_limbs,
                    int n, u64 *out);
// uniform residues drawn coefficient by coefficient (two stream words each):
// the regenerable part of seeded ciphertexts (purpose kSeededPurpose)
void sample_uniform_wide(u64 seed, u64 purpose, u64 index, const u64 *primes, int n_limbs,
                         int n, u64 *out);
constexpr u64 kSeededPurpose = 6;

// CKKS encoding (canonical embedding) in FP64: out [level+1][N]
void encode(int log_n, const double *slots, int n_slots, double scale, const u64 *primes,
            int n_limbs, u64 *out);
// decode from centred integer coefficients (as doubles already divided by scale)
void decode(int log_n, const double *coef, double *slots_out);
double round_half_away(double x);
}  // namespace hm

// ------------------------------------------------------------------ device tables
struct PrimeC;  // modarith.cuh

struct ConvTab {
    // approximate base conversion from n_in primes to n_out primes (device)
    int n_in, n_out;
    int in_p[8], in_l[8];     // prime index and limb position of each input
    int out_p[72], out_l[72]; // prime index and limb position of each output
    u64 hinv[8], hinv_s[8];   // (B/b_k)^-1 mod b_k and its Shoup companion
    u64 hmod[8][72];          // (B/b_k) mod out prime, Montgomery form, 30-bit halves (lo | hi << 32)
    u64 negb[72];             // -B mod out prime, same form (the centred conversion's correction)
};

// kernel launch configurations that compute the same words and differ in
// speed only; the batched form tunes them per shape (defaults: the
// configurations measured best on the benchmark layer)
struct Tune {
    int ntt_cols = 8;      // N = 2^16 NTT pass A: columns per CTA (8 or 16)
    int ntt_rows = 8;      // N = 2^16 NTT pass B: rows per CTA (8 or 16)
    int ntt_tw = 0;        // N = 2^16 NTT twiddles: 0 = held in registers per round (3 CTAs of
                           // 256 threads per SM), 1 = loaded where used (4 per SM)
    int ks_split = 0;      // key switch registers: 0 = launch bounds by digit count, 1 = one CTA per
                           // SM fewer, 2 = key words parked in shared memory (one CTA more)
    int ks_cols = 1;       // key switch: launches the columns are split over (1 or 2)
    int modup_fused = 1;   // N = 2^16 ModUp: 1 = conversion fused into the digits' first NTT pass
    int moddown_fused = 0; // N = 2^16 ModDown + rescale: 1 = conversion fused into the first NTT pass
    int gmac_groups = 7;   // group MAC: outputs from which a CTA runs three thread groups
    int gmac_regs = 1;     // group MAC: 1 = registers for 3 CTAs of 384 threads per SM, 0 = for 2
    int kara = 1;          // group MAC, split products below 2^46: 1 = three products
                           // (Karatsuba), 0 = four
    bool operator==(const Tune &o) const
    {
        return ntt_cols == o.ntt_cols && ntt_rows == o.ntt_rows && ntt_tw == o.ntt_tw &&
               ks_split == o.ks_split && ks_cols == o.ks_cols && modup_fused == o.modup_fused &&
               moddown_fused == o.moddown_fused && gmac_groups == o.gmac_groups &&
               gmac_regs == o.gmac_regs && kara == o.kara;
    }
};

struct fg_ctx {
    Tune tune;                   // launch configurations in use
    Tune batch_tune;             // ... inside batched calls (chosen by timing)
    bool batch_tuned = false;
    std::vector<double> tune_ms; // the batch's time under each configuration tried
    // parameters
    int log_n = 0, n = 0, slots = 0;
    int nq = 0, np = 0, alpha = 0;
    double log_scale = 0, scale = 0;
    std::vector<u64> primes;     // q_0..q_L then p_0..p_{K-1}
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;

    // device constants
    PrimeC *d_primes = nullptr;       // [nq+np]
    void *d_fwd = nullptr;            // ulonglong2 [nq+np][N] (psi^brv(i), Shoup)
    void *d_inv = nullptr;            // ulonglong2 [nq+np][N]
    // N = 2^16: the twiddles of the row stages 12..15 (forward) and of the
    // inverse's first four row stages, laid out [row][stage group][column]
    // so that the 16 threads of a row read 16 consecutive entries
    void *d_fwd_rows = nullptr;       // ulonglong2 [nq+np][256][15][16]
    void *d_inv_rows = nullptr;
    u64 *d_ninv = nullptr;            // [nq+np][2] N^-1 and Shoup
    u64 *d_pmodq = nullptr;           // [nq][2] P mod q_i and Shoup
    std::vector<u64> h_qneg, h_r2, h_ones;

    // cached RNS constant tables, keyed by (kind, level, digit)
    std::map<std::tuple<int, int, int>, ConvTab *> conv_tabs;
    std::map<int, u64 *> rescale_tabs;   // level -> [level][2] q_l^-1 mod q_i + Shoup
    std::map<int, u64 *> pinv_tabs;      // level -> [level+1][2] P^-1 mod q_i + Shoup
    std::map<int, u64 *> modup_scale_tabs;   // level -> [level+1][2] N^-1 (D_j/q_i)^-1 mod q_i + Shoup
    std::map<int, u64 *> moddown_scale_tabs; // level -> [E][2]: limb l N^-1, special k N^-1 (P/p_k)^-1
    std::map<int, u64 *> mdr_tabs;       // level -> [level][2] (P q_l)^-1 mod q_i + Shoup
    std::map<int, u64 *> mdr_half_tabs;  // level -> [level+1] P (q_l - 1)/2 mod q_i (rounded rescale)

    // instrumentation: kernel launch count, and CUDA-event timing of every
    // launch of one kernel class with its algorithmic bytes
    int64_t launches = 0;
    std::string time_class;
    struct Timed {
        cudaEvent_t a, b;
        double bytes;
    };
    std::vector<Timed> timed;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_next = 0;
    cudaEvent_t event();

    // workspace (grow-only arena of named device buffers); names are
    // prefixed with ws_prefix, which batched execution sets per stream
    std::map<std::string, std::pair<void *, size_t>> ws;
    std::string ws_prefix;
    size_t table_bytes = 0;

    // batched execution: streams for layers in flight at once, fork/join
    // events, and the CUDA graph of the last batch with its arguments
    std::vector<cudaStream_t> pool;
    std::vector<cudaEvent_t> pool_events;
    cudaStream_t batch_stream = nullptr;   // the batch's own origin (capturable)
    // host inputs: copied in chunks on their own stream, each chunk's part of
    // the combination starting when the chunk has arrived
    // (one copy stream and its events per workspace prefix, so that layers
    // in flight on different streams copy independently)
    struct CopyRes {
        cudaStream_t st = nullptr;
        std::vector<cudaEvent_t> ev;       // per chunk arrived, then "layer started"
        cudaEvent_t free_ev = nullptr;     // the previous layer has read its staged inputs
        bool have_free = false;            // free_ev was recorded in this batch pass
    };
    std::map<std::string, CopyRes> copies;
    bool in_batch = false;                 // layers of a batch pass are being enqueued
    const uint64_t *batch_seeds = nullptr; // seeded batch: query q's inputs are c0 parts of seeds[q]
    struct BatchGraph {
        std::vector<const void *> args;   // plans, inputs, outputs
        int streams = 0;
        cudaGraphExec_t exec = nullptr;
        int64_t launches = 0;
    } batch;

    int L() const { return nq - 1; }
    int ext(int level) const { return level + 1 + np; }
    int n_digits(int level) const { return (level + 1 + alpha - 1) / alpha; }
    // prime index of extended limb i at level l
    int ext_prime(int level, int i) const { return i <= level ? i : nq + (i - level - 1); }
    void *buf(const std::string &name, size_t bytes);
    const ConvTab *modup_tabs(int level);   // device array, one per digit
    const ConvTab *moddown_tab(int level);
    const u64 *rescale_tab(int level);
    const u64 *pinv_tab(int level);
    const u64 *modup_scale_tab(int level);
    const u64 *moddown_scale_tab(int level);
    const u64 *moddown_rescale_tab(int level);
    const u64 *moddown_rescale_half_tab(int level);
};

struct KeyDev {
    int32_t amount;   // k mod M
    uint32_t galois;
    u64 *d = nullptr; // [beta_L][2][L+1+K][N], NTT domain, Montgomery form
};

struct fg_keys {
    fg_ctx *ctx = nullptr;
    std::map<int32_t, KeyDev> keys;   // amount -> key
    const KeyDev &get(int32_t amount) const;
};

// ------------------------------------------------------------------ plan
struct TermC {
    int src, k, dst, mask;
};
struct GroupC {
    int bit_lo, n_bits, level, n_in, n_out;
    std::vector<std::pair<int, int>> rots;   // (src lane, k)
    std::vector<TermC> terms;
};
struct MaskC {
    int level;
    std::vector<int32_t> slots;   // sorted
    std::vector<double> values;
    u64 *d = nullptr;             // [level+1][N] NTT domain, Montgomery form
};

struct fg_plan {
    fg_ctx *ctx = nullptr;
    int N = 0, M = 0, t = 1, B = 0, V = 0, F = 0, Fp = 0;
    int in_level = 0, out_level = 0, radix_bits = 0, aoo = 1;
    std::vector<int32_t> perm;
    std::vector<i64> comb_consts;          // t == 1: [F][Fp]
    std::vector<std::vector<int>> comb_masks;   // t > 1: [ceil(F/t)][Fp]
    std::vector<int> comb_rots;
    std::vector<GroupC> groups;
    std::vector<MaskC> masks;
    u64 *d_comb = nullptr;                 // t == 1: [in_level+1][F][Fp] Montgomery constants
    int max_lanes = 1;
    int n_copies = 0;                      // Inter-CA: neighbour copies (masks 0..n_copies-1)
};

// ------------------------------------------------------------------ kernels
namespace kern {
// CUDA events around the launches of one kernel class when the context times it
struct KTimer {
    fg_ctx *ctx;
    bool on;
    cudaEvent_t a = nullptr;
    double bytes;
    KTimer(fg_ctx *c, const char *cls, double alg_bytes);
    ~KTimer();
};
// rows x per_row limbs: limb (r, c) at base + (r * stride + c) * N, reduced
// modulo prime pidx[c] (pidx[c] < 0: the limb is left alone)
struct LimbSet {
    u64 *base;
    int stride;
    int per_row;
    int rows;
    std::vector<int> pidx;
};
// negacyclic NTT (forward: natural -> private bit-reversed order), src -> dst
void ntt_fwd(fg_ctx *ctx, const LimbSet &src, const LimbSet &dst);
void ntt_inv(fg_ctx *ctx, const LimbSet &src, const LimbSet &dst);

// contiguous [count][N] limbs, limb c modulo prime pidx[c % pidx.size()]
void to_mont(fg_ctx *ctx, u64 *data, int count, const std::vector<int> &pidx);
void from_mont(fg_ctx *ctx, u64 *data, int count, const std::vector<int> &pidx);
void pointwise(fg_ctx *ctx, const u64 *a, const u64 *b, u64 *c, int count,
               const std::vector<int> &pidx);
void add(fg_ctx *ctx, const u64 *a, const u64 *b, u64 *c, int count, const std::vector<int> &pidx);
void neg(fg_ctx *ctx, const u64 *a, u64 *c, int count, const std::vector<int> &pidx);
// c = a * s[c % period] with d_scal = (w, w') pairs per limb column
void scalar(fg_ctx *ctx, const u64 *a, u64 *c, int count, const std::vector<int> &pidx,
            const u64 *d_scal);
// X -> X^g on NTT-domain limbs (same index map for every prime)
void automorphism(fg_ctx *ctx, const u64 *a, u64 *c, int nlimbs, uint32_t g);
void small_to_res(fg_ctx *ctx, const int8_t *e, u64 *out, int n_limbs, const int *d_pidx);
void copy_limbs(fg_ctx *ctx, const u64 *src, int src_ls, u64 *dst, int dst_ls, int npoly, int nl);
// seeded ciphertexts index0 .. index0 + ncols - 1 at level nl - 1 into
// ct + c * ct_pitch ([2][nl][N]) on stream st: the uniform part regenerated,
// c0 copied from c0 + c * nl * N when c0 is not null (else already in place)
void expand_uniform(fg_ctx *ctx, cudaStream_t st, u64 *ct, size_t ct_pitch, const u64 *c0, int ncols,
                    int nl, u64 seed, u64 index0);

// combination: Z[j][p][i] = sum_f c[i][f][j] X[f][p][i], coefficient domain;
// X: [F][2][level+1][N], consts: [level+1][F][Fp] Montgomery form, Z limb stride z_ls
void comb_const_mac(fg_ctx *ctx, const u64 *X, int F, int Fp, int level, const u64 *consts,
                    u64 *Z, int z_ls, int fb = 0, int fe = -1, bool accumulate = false);
// rescale by q_level, coefficient domain, npoly polys with limb strides
void rescale_coef(fg_ctx *ctx, const u64 *in, int in_ls, u64 *out, int out_ls, int npoly,
                  int level);
// rescale by q_level in the NTT domain, in place (limbs 0..level-1 remain)
void rescale_ntt(fg_ctx *ctx, u64 *ct, int ls, int npoly, int level);

// ModUp of the c1 parts of ncol ciphertexts (NTT domain, limb stride ls) at
// `level`: digits [ncol][beta][E][N], NTT domain, own-digit limbs not written
void modup(fg_ctx *ctx, const u64 *lane, int ls, int ncol, int level, u64 *digits);
struct Dest {
    u64 *out;          // accumulator ciphertexts (limb stride out_ls)
    const u64 *mask;   // [level+1][N] NTT domain, Montgomery form; null = store R
};
// R = Rot(lane, k) from the hoisted digits; every destination gets mask (x) R
void rotate_mac(fg_ctx *ctx, const KeyDev &key, const u64 *lane, int ls, int ncol, int level,
                const u64 *digits, const std::vector<Dest> &dests, int out_ls);
// every destination gets mask (x) lane
struct GroupSource {
    const u64 *u;      // rotation: key-switch output [ncol][2][E][N]; kept lane: nullptr
    const u64 *lane;   // the source lane
    uint32_t galois;
    int t0, t1;        // its terms (indices into the term list)
};
// one SpIntra-CA group's outputs in the extended basis (see k_group_mac);
// a launch takes at most kGmacSrc sources and kGmacTerms terms
constexpr int kGmacSrc = 36;
constexpr int kGmacTerms = 300;
void group_mac(fg_ctx *ctx, const std::vector<GroupSource> &srcs, const std::vector<Dest> &terms,
               const std::vector<int> &term_dest, const std::vector<u64 *> &outs, bool accumulate,
               int ncol, int level, int ls);
// key-switch outputs u_r = sum_d D_d(sigma_r) evk_r + P phi_r(c0) of several
// rotations r of one lane (extended basis, NTT domain, [ncol][2][E][N] each)
void ks_multi(fg_ctx *ctx, const std::vector<const KeyDev *> &keys, const std::vector<u64 *> &us,
              const u64 *lane, int ls, int ncol, int level, const u64 *digits);
// ModDown of an extended-basis sum to Q, then the rescale by q_level, into a
// lane (limbs 0..level-1); ext is scratch and is overwritten
void moddown_rescale_to_lane(fg_ctx *ctx, u64 *ext, int ncol, int level, u64 *out, int ls);
// residues mod the special primes from limb 0 (centred): out [np][N]
void lift_special(fg_ctx *ctx, const u64 *limb0, u64 *out);
void stay_mac(fg_ctx *ctx, const u64 *lane, int ls, int ncol, int level,
              const std::vector<Dest> &dests, int out_ls);
}  // namespace kern

// ------------------------------------------------------------------ planner
namespace planner {
int choose_t(int F, int n, int V, int Fp, int M);
void build(fg_plan &pl, const fg_ctx &ctx, const int32_t *row_ptr, const int32_t *col,
           const double *val, int V, const double *W, int F, int Fp, const int32_t *perm,
           const fg_plan_opts &opts);
// Inter-CA plan: combination constants of W, then one mask per neighbour
// copy k holding wts[v][k] at slot perm[v]
void build_inter(fg_plan &pl, const fg_ctx &ctx, const int32_t *nbr, const double *wts, int V,
                 int n, const double *W, int F, int Fp, const int32_t *perm, const fg_plan_opts &opts);
// aggregation mode of one layer from the SpIntra-CA plan's counts (see planner.cpp)
void select_mode(const fg_plan &pl, int layer, int n_copies, const double lat[3], double max_inter_cts,
                 int *mode, double cost[2], int64_t counts[4]);
}  // namespace planner
