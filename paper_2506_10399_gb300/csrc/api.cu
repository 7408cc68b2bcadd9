// api.cu -- the C ABI of include/ficgcn.h: contexts, keys, client-side
// encryption, plans and the encrypted A-hat X W layer.
#include <omp.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "fg_internal.h"
#include "modarith.cuh"

// ====================================================================== helpers
// message of the last failed call that has no context (fg_last_error(NULL))
std::string g_create_err = "no context";

namespace {

constexpr int kMaxQ = 60, kMaxP = 7;   // the centred ModDown conversion takes one extra product term

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// a device view of a caller buffer: the buffer itself, or a staged copy
const u64 *stage_in(fg_ctx *ctx, const u64 *p, size_t words, const char *name)
{
    FG_CHECK(p != nullptr, FG_EINVAL, "null buffer");
    if (is_device_ptr(p)) return p;
    u64 *d = (u64 *)ctx->buf(name, words * 8);
    CUDA_TRY(cudaMemcpyAsync(d, p, words * 8, cudaMemcpyHostToDevice, ctx->stream));
    return d;
}

void stage_out(fg_ctx *ctx, u64 *dst, const u64 *dev, size_t words)
{
    FG_CHECK(dst != nullptr, FG_EINVAL, "null output buffer");
    if (dst != dev)
        CUDA_TRY(cudaMemcpyAsync(dst, dev, words * 8, cudaMemcpyDefault, ctx->stream));
}

void sync(fg_ctx *ctx) { CUDA_TRY(cudaStreamSynchronize(ctx->stream)); }

std::vector<int> iota(int n, int start = 0)
{
    std::vector<int> v(n);
    for (int i = 0; i < n; i++) v[i] = start + i;
    return v;
}

// 64-bit FNV-1a over 8-byte words (little-endian), tail bytes zero-padded
u64 checksum(const uint8_t *p, size_t len)
{
    u64 h = 0xcbf29ce484222325ull;
    size_t i = 0;
    for (; i + 8 <= len; i += 8) {
        u64 w;
        memcpy(&w, p + i, 8);
        h = (h ^ w) * 0x100000001b3ull;
    }
    if (i < len) {
        u64 w = 0;
        memcpy(&w, p + i, len - i);
        h = (h ^ w) * 0x100000001b3ull;
    }
    return h;
}

struct Writer {
    std::vector<uint8_t> b;
    template <class T> void put(const T &v)
    {
        const uint8_t *p = (const uint8_t *)&v;
        b.insert(b.end(), p, p + sizeof(T));
    }
};

struct Reader {
    const uint8_t *p;
    size_t len, off = 0;
    template <class T> T get()
    {
        FG_CHECK(off + sizeof(T) <= len, FG_EKEY, "blob truncated");
        T v;
        memcpy(&v, p + off, sizeof(T));
        off += sizeof(T);
        return v;
    }
};

const char kSkMagic[8] = {'F', 'G', 'S', 'K', '0', '0', '0', '1'};
const char kEvkMagic[8] = {'F', 'G', 'E', 'V', 'K', '0', '0', '1'};

void *blob_copy(const std::vector<uint8_t> &b)
{
    void *p = malloc(b.size());
    FG_CHECK(p != nullptr, FG_EOOM, "host allocation failed");
    memcpy(p, b.data(), b.size());
    return p;
}

}  // namespace

// ====================================================================== context
void *fg_ctx::buf(const std::string &name0, size_t bytes)
{
    const std::string name = ws_prefix + name0;
    auto it = ws.find(name);
    if (it != ws.end() && it->second.second >= bytes) return it->second.first;
    if (it != ws.end()) {
        CUDA_TRY(cudaDeviceSynchronize());   // any stream may still use it
        CUDA_TRY(cudaFree(it->second.first));
        ws.erase(it);
    }
    void *p = nullptr;
    CUDA_TRY(cudaMalloc(&p, std::max<size_t>(bytes, 256)));
    ws[name] = {p, bytes};
    return p;
}

extern "C" int fg_ctx_release_workspace(fg_ctx *ctx)
{
    if (!ctx) return FG_EINVAL;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        ctx->err = "device synchronisation failed";
        return FG_ECUDA;
    }
    for (auto &kv : ctx->ws) cudaFree(kv.second.first);
    ctx->ws.clear();
    if (ctx->batch.exec) {   // a captured batch refers to the workspace
        cudaGraphExecDestroy(ctx->batch.exec);
        ctx->batch.exec = nullptr;
        ctx->batch.args.clear();
    }
    return FG_OK;
}

cudaEvent_t fg_ctx::event()
{
    if (ev_next == ev_pool.size()) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreate(&e));
        ev_pool.push_back(e);
    }
    return ev_pool[ev_next++];
}

static ConvTab make_conv(const fg_ctx &c, const std::vector<int> &in_p, const std::vector<int> &in_l,
                         const std::vector<int> &out_p, const std::vector<int> &out_l)
{
    ConvTab T;
    memset(&T, 0, sizeof(T));
    FG_CHECK(in_p.size() <= 8 && out_p.size() <= 72, FG_EINVAL, "conversion table too wide");
    T.n_in = (int)in_p.size();
    T.n_out = (int)out_p.size();
    for (int k = 0; k < T.n_in; k++) {
        const u64 bk = c.primes[in_p[k]];
        u64 h = 1;   // (B / b_k) mod b_k
        for (int j = 0; j < T.n_in; j++)
            if (j != k) h = hm::mulmod(h, c.primes[in_p[j]] % bk, bk);
        T.in_p[k] = in_p[k];
        T.in_l[k] = in_l[k];
        T.hinv[k] = hm::invmod(h, bk);
        T.hinv_s[k] = hm::shoup(T.hinv[k], bk);
        for (int t = 0; t < T.n_out; t++) {
            const u64 p = c.primes[out_p[t]];
            u64 hp = 1;   // (B / b_k) mod p
            for (int j = 0; j < T.n_in; j++)
                if (j != k) hp = hm::mulmod(hp, c.primes[in_p[j]] % p, p);
            const u64 hm_ = hm::to_mont(hp, p);
            T.hmod[k][t] = (hm_ & 0x3FFFFFFFull) | ((hm_ >> 30) << 32);   // 30-bit halves
        }
    }
    for (int t = 0; t < T.n_out; t++) {
        T.out_p[t] = out_p[t];
        T.out_l[t] = out_l[t];
        const u64 p = c.primes[out_p[t]];
        u64 B = 1;   // B mod p
        for (int j = 0; j < T.n_in; j++) B = hm::mulmod(B, c.primes[in_p[j]] % p, p);
        const u64 nb = hm::to_mont((p - B) % p, p);
        T.negb[t] = (nb & 0x3FFFFFFFull) | ((nb >> 30) << 32);
    }
    return T;
}

const ConvTab *fg_ctx::modup_tabs(int level)
{
    auto key = std::make_tuple(0, level, 0);
    auto it = conv_tabs.find(key);
    if (it != conv_tabs.end()) return it->second;
    const int beta = n_digits(level), E = ext(level);
    std::vector<ConvTab> h(beta);
    for (int d = 0; d < beta; d++) {
        std::vector<int> ip, il, op, ol;
        for (int i = d * alpha; i < std::min((d + 1) * alpha, level + 1); i++) {
            ip.push_back(i);
            il.push_back(i);
        }
        for (int i = 0; i < E; i++) {
            if (i <= level && i / alpha == d) continue;
            op.push_back(ext_prime(level, i));
            ol.push_back(i);
        }
        h[d] = make_conv(*this, ip, il, op, ol);
    }
    ConvTab *d = nullptr;
    CUDA_TRY(cudaMalloc(&d, sizeof(ConvTab) * beta));
    CUDA_TRY(cudaMemcpy(d, h.data(), sizeof(ConvTab) * beta, cudaMemcpyHostToDevice));
    table_bytes += sizeof(ConvTab) * beta;
    conv_tabs[key] = d;
    return d;
}

const ConvTab *fg_ctx::moddown_tab(int level)
{
    auto key = std::make_tuple(1, level, 0);
    auto it = conv_tabs.find(key);
    if (it != conv_tabs.end()) return it->second;
    std::vector<int> ip, il, op, ol;
    for (int k = 0; k < np; k++) {
        ip.push_back(nq + k);
        il.push_back(level + 1 + k);
    }
    for (int i = 0; i <= level; i++) {
        op.push_back(i);
        ol.push_back(i);
    }
    // the centred conversion adds one product (c times -P) to the K inputs
    FG_CHECK(np <= 7, FG_EINVAL, "ModDown conversion: at most 7 special primes");
    ConvTab h = make_conv(*this, ip, il, op, ol);
    ConvTab *d = nullptr;
    CUDA_TRY(cudaMalloc(&d, sizeof(ConvTab)));
    CUDA_TRY(cudaMemcpy(d, &h, sizeof(ConvTab), cudaMemcpyHostToDevice));
    table_bytes += sizeof(ConvTab);
    conv_tabs[key] = d;
    return d;
}

const u64 *fg_ctx::rescale_tab(int level)
{
    auto it = rescale_tabs.find(level);
    if (it != rescale_tabs.end()) return it->second;
    std::vector<u64> h(2 * std::max(level, 1));
    const u64 ql = primes[level];
    for (int i = 0; i < level; i++) {
        const u64 q = primes[i];
        h[2 * i] = hm::invmod(ql % q, q);
        h[2 * i + 1] = hm::shoup(h[2 * i], q);
    }
    u64 *d = nullptr;
    CUDA_TRY(cudaMalloc(&d, h.size() * 8));
    CUDA_TRY(cudaMemcpy(d, h.data(), h.size() * 8, cudaMemcpyHostToDevice));
    rescale_tabs[level] = d;
    return d;
}

const u64 *fg_ctx::pinv_tab(int level)
{
    auto it = pinv_tabs.find(level);
    if (it != pinv_tabs.end()) return it->second;
    std::vector<u64> h(2 * (level + 1));
    for (int i = 0; i <= level; i++) {
        const u64 q = primes[i];
        u64 P = 1;
        for (int k = 0; k < np; k++) P = hm::mulmod(P, primes[nq + k] % q, q);
        h[2 * i] = hm::invmod(P, q);
        h[2 * i + 1] = hm::shoup(h[2 * i], q);
    }
    u64 *d = nullptr;
    CUDA_TRY(cudaMalloc(&d, h.size() * 8));
    CUDA_TRY(cudaMemcpy(d, h.data(), h.size() * 8, cudaMemcpyHostToDevice));
    pinv_tabs[level] = d;
    return d;
}

// per limb i of q_0..q_level in digit D_j: N^-1 (D_j / q_i)^-1 mod q_i, so
// that an inverse NTT scaled by it yields the base conversion's inputs
// y_i = [x_i (D_j / q_i)^-1]_{q_i} directly
const u64 *fg_ctx::modup_scale_tab(int level)
{
    auto it = modup_scale_tabs.find(level);
    if (it != modup_scale_tabs.end()) return it->second;
    std::vector<u64> h(2 * (level + 1));
    for (int i = 0; i <= level; i++) {
        const u64 q = primes[i];
        const int d = i / alpha;
        u64 hd = 1;
        for (int j = d * alpha; j < std::min((d + 1) * alpha, level + 1); j++)
            if (j != i) hd = hm::mulmod(hd, primes[j] % q, q);
        const u64 ninv = hm::invmod((u64)n % q, q);
        h[2 * i] = hm::mulmod(ninv, hm::invmod(hd, q), q);
        h[2 * i + 1] = hm::shoup(h[2 * i], q);
    }
    u64 *dptr = nullptr;
    CUDA_TRY(cudaMalloc(&dptr, h.size() * 8));
    CUDA_TRY(cudaMemcpy(dptr, h.data(), h.size() * 8, cudaMemcpyHostToDevice));
    modup_scale_tabs[level] = dptr;
    return dptr;
}

// per extended limb of level l (positions 0..E-1): at position l, N^-1 mod
// q_l; at the special limb of p_k, N^-1 (P / p_k)^-1 mod p_k (an inverse NTT
// scaled by it yields the centred conversion's inputs before centring);
// other positions unused
const u64 *fg_ctx::moddown_scale_tab(int level)
{
    auto it = moddown_scale_tabs.find(level);
    if (it != moddown_scale_tabs.end()) return it->second;
    const int E = ext(level);
    std::vector<u64> h(2 * E, 0);
    {
        const u64 q = primes[level];
        h[2 * level] = hm::invmod((u64)n % q, q);
        h[2 * level + 1] = hm::shoup(h[2 * level], q);
    }
    for (int k = 0; k < np; k++) {
        const u64 p = primes[nq + k];
        u64 hk = 1;
        for (int j = 0; j < np; j++)
            if (j != k) hk = hm::mulmod(hk, primes[nq + j] % p, p);
        const int i = level + 1 + k;
        h[2 * i] = hm::mulmod(hm::invmod((u64)n % p, p), hm::invmod(hk, p), p);
        h[2 * i + 1] = hm::shoup(h[2 * i], p);
    }
    u64 *dptr = nullptr;
    CUDA_TRY(cudaMalloc(&dptr, h.size() * 8));
    CUDA_TRY(cudaMemcpy(dptr, h.data(), h.size() * 8, cudaMemcpyHostToDevice));
    moddown_scale_tabs[level] = dptr;
    return dptr;
}

const u64 *fg_ctx::moddown_rescale_tab(int level)
{
    auto it = mdr_tabs.find(level);
    if (it != mdr_tabs.end()) return it->second;
    std::vector<u64> h(2 * std::max(level, 1));
    for (int i = 0; i < level; i++) {
        const u64 q = primes[i];
        u64 Pq = primes[level] % q;
        for (int k = 0; k < np; k++) Pq = hm::mulmod(Pq, primes[nq + k] % q, q);
        h[2 * i] = hm::invmod(Pq, q);
        h[2 * i + 1] = hm::shoup(h[2 * i], q);
    }
    u64 *d = nullptr;
    CUDA_TRY(cudaMalloc(&d, h.size() * 8));
    CUDA_TRY(cudaMemcpy(d, h.data(), h.size() * 8, cudaMemcpyHostToDevice));
    mdr_tabs[level] = d;
    return d;
}

// the offset of the rounded rescale that follows a ModDown, seen before the
// division by P: H = P (q_l - 1) / 2, mod q_0..q_l
const u64 *fg_ctx::moddown_rescale_half_tab(int level)
{
    auto it = mdr_half_tabs.find(level);
    if (it != mdr_half_tabs.end()) return it->second;
    std::vector<u64> h(level + 1);
    const u64 hl = (primes[level] - 1) / 2;
    for (int i = 0; i <= level; i++) {
        const u64 q = primes[i];
        u64 P = 1;
        for (int k = 0; k < np; k++) P = hm::mulmod(P, primes[nq + k] % q, q);
        h[i] = hm::mulmod(P, hl % q, q);
    }
    u64 *d = nullptr;
    CUDA_TRY(cudaMalloc(&d, h.size() * 8));
    CUDA_TRY(cudaMemcpy(d, h.data(), h.size() * 8, cudaMemcpyHostToDevice));
    mdr_half_tabs[level] = d;
    return d;
}

const KeyDev &fg_keys::get(int32_t amount) const
{
    auto it = keys.find(amount);
    FG_CHECK(it != keys.end(), FG_EKEY, "no rotation key for amount " + std::to_string(amount));
    return it->second;
}

// extra per-context state kept out of the shared header
namespace {
struct SkCache {
    u64 sum = 0;
    u64 *d = nullptr;   // s in the NTT domain over all primes [nq+np][N]
};
std::map<const fg_ctx *, SkCache> g_sk;
std::map<const fg_ctx *, u64 *> g_pmodq;     // [nq][2] P mod q_i, Shoup
std::map<const fg_ctx *, int *> g_pidx_all;  // [nq+np] 0..nq+np-1

// parse a secret-key blob and return s in the NTT domain on the device
const u64 *secret_ntt(fg_ctx *ctx, const void *blob, size_t len)
{
    FG_CHECK(blob != nullptr, FG_EINVAL, "null secret key");
    const uint8_t *p = (const uint8_t *)blob;
    const size_t want = 8 + 8 + (size_t)ctx->n + 8;
    FG_CHECK(len == want && memcmp(p, kSkMagic, 8) == 0, FG_EKEY, "not a secret-key blob");
    uint32_t log_n;
    memcpy(&log_n, p + 8, 4);
    FG_CHECK((int)log_n == ctx->log_n, FG_EKEY, "secret key for another ring degree");
    u64 sum;
    memcpy(&sum, p + want - 8, 8);
    FG_CHECK(checksum(p, want - 8) == sum, FG_EKEY, "secret-key checksum mismatch");
    SkCache &c = g_sk[ctx];
    if (c.d && c.sum == sum) return c.d;
    const int KL = ctx->nq + ctx->np, N = ctx->n;
    if (!c.d) CUDA_TRY(cudaMalloc(&c.d, (size_t)KL * N * 8));
    int8_t *ds = (int8_t *)ctx->buf("sk_small", N);
    CUDA_TRY(cudaMemcpyAsync(ds, p + 16, N, cudaMemcpyHostToDevice, ctx->stream));
    kern::small_to_res(ctx, ds, c.d, KL, g_pidx_all[ctx]);
    kern::LimbSet s{c.d, KL, KL, 1, iota(KL)};
    kern::ntt_fwd(ctx, s, s);
    sync(ctx);
    c.sum = sum;
    return c.d;
}

// c = (-a s + m + e, a) at `level`; pt and out on the device
void encrypt_dev(fg_ctx *ctx, const u64 *S, u64 seed, u64 index, const u64 *pt, int level,
                 u64 *out, const u64 *host_a, const int8_t *host_e)
{
    const int N = ctx->n, nl = level + 1;
    std::vector<int> pid = iota(nl);
    u64 *c0 = out, *c1 = out + (size_t)nl * N;
    CUDA_TRY(cudaMemcpyAsync(c1, host_a, (size_t)nl * N * 8, cudaMemcpyHostToDevice, ctx->stream));
    u64 *t = (u64 *)ctx->buf("enc_t", (size_t)nl * N * 8);
    kern::LimbSet src{c1, nl, nl, 1, pid}, dst{t, nl, nl, 1, pid};
    kern::ntt_fwd(ctx, src, dst);
    kern::pointwise(ctx, t, S, t, nl, pid);
    kern::ntt_inv(ctx, dst, dst);
    kern::neg(ctx, t, t, nl, pid);
    kern::add(ctx, t, pt, t, nl, pid);
    int8_t *de = (int8_t *)ctx->buf("enc_e", N);
    CUDA_TRY(cudaMemcpyAsync(de, host_e, N, cudaMemcpyHostToDevice, ctx->stream));
    u64 *er = (u64 *)ctx->buf("enc_er", (size_t)nl * N * 8);
    kern::small_to_res(ctx, de, er, nl, g_pidx_all[ctx]);
    kern::add(ctx, t, er, c0, nl, pid);
    sync(ctx);   // host_a / host_e may be reused by the caller
}

// m = c0 + c1 s on the device (coefficient domain)
void decrypt_dev(fg_ctx *ctx, const u64 *S, const u64 *ct, int level, u64 *m)
{
    const int N = ctx->n, nl = level + 1;
    std::vector<int> pid = iota(nl);
    u64 *t = (u64 *)ctx->buf("dec_t", (size_t)nl * N * 8);
    kern::LimbSet src{const_cast<u64 *>(ct) + (size_t)nl * N, nl, nl, 1, pid}, dst{t, nl, nl, 1, pid};
    kern::ntt_fwd(ctx, src, dst);
    kern::pointwise(ctx, t, S, t, nl, pid);
    kern::ntt_inv(ctx, dst, dst);
    kern::add(ctx, t, ct, m, nl, pid);
}

}  // namespace

#define API_TRY try {
#define API_CATCH(ctxp)                                                   \
    }                                                                     \
    catch (const fg_error &e)                                             \
    {                                                                     \
        if (ctxp) (ctxp)->err = e.what();                                 \
        return e.code;                                                    \
    }                                                                     \
    catch (const std::bad_alloc &)                                        \
    {                                                                     \
        if (ctxp) (ctxp)->err = "host allocation failed";                 \
        return FG_EOOM;                                                   \
    }                                                                     \
    catch (const std::exception &e)                                       \
    {                                                                     \
        if (ctxp) (ctxp)->err = e.what();                                 \
        return FG_EINVAL;                                                 \
    }                                                                     \
    return FG_OK;

extern "C" {

int fg_ctx_create(const fg_params *prm, void *cuda_stream, fg_ctx **out)
{
    if (!prm || !out) return FG_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return FG_ENODEV;
    }
    fg_ctx *ctx = new (std::nothrow) fg_ctx;
    if (!ctx) return FG_EOOM;
    try {
        FG_CHECK(prm->log_n >= 10 && prm->log_n <= 16, FG_EINVAL, "log_n must be in [10, 16]");
        FG_CHECK(prm->n_q >= 2 && prm->n_q <= kMaxQ && prm->q_bits, FG_EINVAL, "n_q must be in [2, 60]");
        FG_CHECK(prm->n_p >= 1 && prm->n_p <= kMaxP && prm->p_bits, FG_EINVAL, "n_p must be in [1, 7]");
        FG_CHECK(prm->alpha >= 1 && prm->alpha <= 8, FG_EINVAL, "alpha must be in [1, 8]");
        FG_CHECK(prm->log_scale > 0 && prm->log_scale < 62, FG_EINVAL, "bad log_scale");
        ctx->log_n = prm->log_n;
        ctx->n = 1 << prm->log_n;
        ctx->slots = ctx->n / 2;
        ctx->nq = prm->n_q;
        ctx->np = prm->n_p;
        ctx->alpha = prm->alpha;
        ctx->log_scale = prm->log_scale;
        ctx->scale = std::ldexp(1.0, 0) * std::pow(2.0, prm->log_scale);
        FG_CHECK(ctx->n_digits(ctx->L()) <= 16, FG_EINVAL, "more than 16 key-switching digits");
        std::vector<int> bits(prm->q_bits, prm->q_bits + prm->n_q);
        bits.insert(bits.end(), prm->p_bits, prm->p_bits + prm->n_p);
        ctx->primes = hm::gen_primes(ctx->log_n, bits);
        ctx->stream = (cudaStream_t)cuda_stream;
        CUDA_TRY(cudaGetDevice(&ctx->device));
        const int KL = ctx->nq + ctx->np, N = ctx->n;
        std::vector<PrimeC> pc(KL);
        std::vector<ulonglong2> fwd((size_t)KL * N), inv((size_t)KL * N);
        std::vector<u64> ninv(2 * KL), pw(N), pwi(N);
        for (int k = 0; k < KL; k++) {
            const u64 q = ctx->primes[k];
            pc[k].q = q;
            pc[k].qneg = hm::mont_qneg(q);
            const u64 r = (u64)(((u128)1 << 64) % q);
            pc[k].r2 = hm::mulmod(r, r, q);
            pc[k].one_s = hm::shoup(1, q);
            const u64 psi = hm::find_psi(N, q), psii = hm::invmod(psi, q);
            pw[0] = pwi[0] = 1;
            for (int i = 1; i < N; i++) {
                pw[i] = hm::mulmod(pw[i - 1], psi, q);
                pwi[i] = hm::mulmod(pwi[i - 1], psii, q);
            }
            for (int i = 0; i < N; i++) {
                const int b = hm::bitrev(i, ctx->log_n);
                fwd[(size_t)k * N + i] = make_ulonglong2(pw[b], hm::shoup(pw[b], q));
                inv[(size_t)k * N + i] = make_ulonglong2(pwi[b], hm::shoup(pwi[b], q));
            }
            ninv[2 * k] = hm::invmod((u64)N % q, q);
            ninv[2 * k + 1] = hm::shoup(ninv[2 * k], q);
        }
        CUDA_TRY(cudaMalloc(&ctx->d_primes, sizeof(PrimeC) * KL));
        CUDA_TRY(cudaMalloc(&ctx->d_fwd, sizeof(ulonglong2) * KL * N));
        CUDA_TRY(cudaMalloc(&ctx->d_inv, sizeof(ulonglong2) * KL * N));
        CUDA_TRY(cudaMalloc(&ctx->d_ninv, 16 * KL));
        CUDA_TRY(cudaMemcpy(ctx->d_primes, pc.data(), sizeof(PrimeC) * KL, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(ctx->d_fwd, fwd.data(), sizeof(ulonglong2) * KL * N, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(ctx->d_inv, inv.data(), sizeof(ulonglong2) * KL * N, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(ctx->d_ninv, ninv.data(), 16 * KL, cudaMemcpyHostToDevice));
        ctx->table_bytes = sizeof(PrimeC) * KL + 2 * sizeof(ulonglong2) * KL * N + 16 * KL;
        if (ctx->log_n == 16) {
            // row-stage twiddles for the radix-16 row pass: entry (row r,
            // stage st, group g, column j) = table[2^(12+st) + (r << (4+st)) + (j << st) + g]
            const size_t per = (size_t)256 * 15 * 16;
            std::vector<ulonglong2> fr(KL * per), ir(KL * per);
            for (int k = 0; k < KL; k++)
                for (int r = 0; r < 256; r++)
                    for (int st = 0; st < 4; st++)
                        for (int g = 0; g < (1 << st); g++)
                            for (int j = 0; j < 16; j++) {
                                const size_t src = (size_t)k * N + (1u << (12 + st)) + ((size_t)r << (4 + st)) +
                                                   ((size_t)j << st) + g;
                                const size_t dst = (size_t)k * per + ((size_t)r * 15 + (1 << st) - 1 + g) * 16 + j;
                                fr[dst] = fwd[src];
                                ir[dst] = inv[src];
                            }
            CUDA_TRY(cudaMalloc(&ctx->d_fwd_rows, sizeof(ulonglong2) * KL * per));
            CUDA_TRY(cudaMalloc(&ctx->d_inv_rows, sizeof(ulonglong2) * KL * per));
            CUDA_TRY(cudaMemcpy(ctx->d_fwd_rows, fr.data(), sizeof(ulonglong2) * KL * per, cudaMemcpyHostToDevice));
            CUDA_TRY(cudaMemcpy(ctx->d_inv_rows, ir.data(), sizeof(ulonglong2) * KL * per, cudaMemcpyHostToDevice));
            ctx->table_bytes += 2 * sizeof(ulonglong2) * KL * per;
        }
        // P mod q_i (Shoup) and the identity prime-index list
        std::vector<u64> pm(2 * ctx->nq);
        for (int i = 0; i < ctx->nq; i++) {
            const u64 q = ctx->primes[i];
            u64 P = 1;
            for (int k = 0; k < ctx->np; k++) P = hm::mulmod(P, ctx->primes[ctx->nq + k] % q, q);
            pm[2 * i] = P;
            pm[2 * i + 1] = hm::shoup(P, q);
        }
        u64 *dpm = nullptr;
        CUDA_TRY(cudaMalloc(&dpm, pm.size() * 8));
        CUDA_TRY(cudaMemcpy(dpm, pm.data(), pm.size() * 8, cudaMemcpyHostToDevice));
        g_pmodq[ctx] = dpm;
        ctx->d_pmodq = dpm;
        std::vector<int> ids = iota(KL);
        int *dpi = nullptr;
        CUDA_TRY(cudaMalloc(&dpi, ids.size() * sizeof(int)));
        CUDA_TRY(cudaMemcpy(dpi, ids.data(), ids.size() * sizeof(int), cudaMemcpyHostToDevice));
        g_pidx_all[ctx] = dpi;
    } catch (const fg_error &e) {
        int code = e.code;
        g_create_err = e.what();
        fg_ctx_destroy(ctx);
        return code;
    } catch (const std::exception &e) {
        g_create_err = e.what();
        fg_ctx_destroy(ctx);
        return FG_EOOM;
    }
    *out = ctx;
    return FG_OK;
}

int fg_ctx_destroy(fg_ctx *ctx)
{
    if (!ctx) return FG_OK;
    cudaStreamSynchronize(ctx->stream);
    for (cudaStream_t st : ctx->pool) cudaStreamSynchronize(st);
    if (ctx->batch_stream) cudaStreamSynchronize(ctx->batch_stream);
    for (auto &kv : ctx->copies)
        if (kv.second.st) cudaStreamSynchronize(kv.second.st);
    cudaFree(ctx->d_primes);
    cudaFree(ctx->d_fwd);
    cudaFree(ctx->d_inv);
    cudaFree(ctx->d_fwd_rows);
    cudaFree(ctx->d_inv_rows);
    cudaFree(ctx->d_ninv);
    for (auto &kv : ctx->conv_tabs) cudaFree(kv.second);
    for (auto &kv : ctx->rescale_tabs) cudaFree(kv.second);
    for (auto &kv : ctx->pinv_tabs) cudaFree(kv.second);
    for (auto &kv : ctx->mdr_tabs) cudaFree(kv.second);
    for (auto &kv : ctx->mdr_half_tabs) cudaFree(kv.second);
    for (auto &kv : ctx->modup_scale_tabs) cudaFree(kv.second);
    for (auto &kv : ctx->moddown_scale_tabs) cudaFree(kv.second);
    for (auto &kv : ctx->ws) cudaFree(kv.second.first);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    if (ctx->batch.exec) cudaGraphExecDestroy(ctx->batch.exec);
    for (cudaStream_t st : ctx->pool) cudaStreamDestroy(st);
    if (ctx->batch_stream) cudaStreamDestroy(ctx->batch_stream);
    for (auto &kv : ctx->copies) {
        if (kv.second.st) cudaStreamDestroy(kv.second.st);
        for (cudaEvent_t e : kv.second.ev) cudaEventDestroy(e);
        if (kv.second.free_ev) cudaEventDestroy(kv.second.free_ev);
    }
    for (cudaEvent_t e : ctx->pool_events) cudaEventDestroy(e);
    auto s = g_sk.find(ctx);
    if (s != g_sk.end()) {
        cudaFree(s->second.d);
        g_sk.erase(s);
    }
    auto pm = g_pmodq.find(ctx);
    if (pm != g_pmodq.end()) {
        cudaFree(pm->second);
        g_pmodq.erase(pm);
    }
    auto pi = g_pidx_all.find(ctx);
    if (pi != g_pidx_all.end()) {
        cudaFree(pi->second);
        g_pidx_all.erase(pi);
    }
    delete ctx;
    return FG_OK;
}

const char *fg_last_error(const fg_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

int fg_ctx_primes(const fg_ctx *ctx, uint64_t *q_out, uint64_t *p_out)
{
    if (!ctx) return FG_EINVAL;
    if (q_out) memcpy(q_out, ctx->primes.data(), 8 * ctx->nq);
    if (p_out) memcpy(p_out, ctx->primes.data() + ctx->nq, 8 * ctx->np);
    return FG_OK;
}

int fg_ctx_device_bytes(const fg_ctx *ctx, size_t *bytes)
{
    if (!ctx || !bytes) return FG_EINVAL;
    size_t b = ctx->table_bytes;
    for (auto &kv : ctx->ws) b += kv.second.second;
    *bytes = b;
    return FG_OK;
}

void fg_free(void *blob) { free(blob); }

int fg_ctx_time_kernels(fg_ctx *ctx, const char *kernel_class)
{
    if (!ctx) return FG_EINVAL;
    API_TRY
    sync(ctx);
    ctx->time_class = kernel_class ? kernel_class : "";
    ctx->timed.clear();
    ctx->ev_next = 0;
    API_CATCH(ctx)
}

int fg_ctx_kernel_times(fg_ctx *ctx, double *ms, int64_t *calls, double *alg_bytes)
{
    if (!ctx || !ms || !calls || !alg_bytes) return FG_EINVAL;
    API_TRY
    sync(ctx);
    double t = 0, b = 0;
    for (auto &r : ctx->timed) {
        float e = 0;
        CUDA_TRY(cudaEventElapsedTime(&e, r.a, r.b));
        t += e;
        b += r.bytes;
    }
    *ms = t;
    *calls = (int64_t)ctx->timed.size();
    *alg_bytes = b;
    ctx->timed.clear();
    ctx->ev_next = 0;
    API_CATCH(ctx)
}

int fg_ctx_launch_count(const fg_ctx *ctx, int64_t *launches)
{
    if (!ctx || !launches) return FG_EINVAL;
    *launches = ctx->launches;
    return FG_OK;
}

// ---------------------------------------------------------------- client side
int fg_keygen(fg_ctx *ctx, uint64_t seed, const int32_t *rot_amounts, int n_rot, int relin,
              void **sk_blob, size_t *sk_len, void **evk_blob, size_t *evk_len)
{
    if (!ctx) return FG_EINVAL;
    API_TRY
    FG_CHECK(sk_blob && sk_len && evk_blob && evk_len, FG_EINVAL, "null output");
    FG_CHECK(n_rot >= 0 && (n_rot == 0 || rot_amounts), FG_EINVAL, "bad rotation list");
    const int N = ctx->n, M = ctx->slots, KL = ctx->nq + ctx->np, L = ctx->L();
    // secret key blob
    std::vector<int8_t> s(N);
    hm::sample_ternary(seed, 1, 0, N, s.data());
    Writer sw;
    sw.b.insert(sw.b.end(), kSkMagic, kSkMagic + 8);
    sw.put<uint32_t>(ctx->log_n);
    sw.put<uint32_t>(0);
    sw.b.insert(sw.b.end(), (uint8_t *)s.data(), (uint8_t *)s.data() + N);
    sw.put<u64>(checksum(sw.b.data(), sw.b.size()));
    const u64 *S = secret_ntt(ctx, sw.b.data(), sw.b.size());
    // distinct amounts mod M
    std::vector<int32_t> am;
    for (int i = 0; i < n_rot; i++) am.push_back(((rot_amounts[i] % M) + M) % M);
    std::sort(am.begin(), am.end());
    am.erase(std::unique(am.begin(), am.end()), am.end());
    am.erase(std::remove(am.begin(), am.end(), 0), am.end());
    if (relin) am.push_back(FG_RELIN);   // last entry: the relinearisation key
    const int beta = ctx->n_digits(L);
    const size_t limb_w = (size_t)N, key_w = (size_t)beta * 2 * KL * N;
    Writer ew;
    ew.b.insert(ew.b.end(), kEvkMagic, kEvkMagic + 8);
    ew.put<uint32_t>(1);
    ew.put<uint32_t>(ctx->log_n);
    ew.put<uint32_t>(ctx->nq);
    ew.put<uint32_t>(ctx->np);
    ew.put<uint32_t>(ctx->alpha);
    ew.put<uint32_t>((uint32_t)am.size());
    for (u64 p : ctx->primes) ew.put<u64>(p);
    std::vector<uint32_t> gal(am.size());
    for (size_t i = 0; i < am.size(); i++) {
        gal[i] = am[i] == FG_RELIN ? 1u : (uint32_t)hm::powmod(5, am[i], 2 * (u64)N);
        ew.put<int32_t>(am[i]);
        ew.put<uint32_t>(gal[i]);
    }
    const size_t data_off = ew.b.size();
    ew.b.resize(data_off + am.size() * key_w * 8 + 8);
    u64 *A = (u64 *)ctx->buf("kg_a", (size_t)KL * N * 8);
    u64 *Bv = (u64 *)ctx->buf("kg_b", (size_t)KL * N * 8);
    u64 *Sg = (u64 *)ctx->buf("kg_sg", (size_t)KL * N * 8);
    u64 *T = (u64 *)ctx->buf("kg_t", (size_t)KL * N * 8);
    u64 *Er = (u64 *)ctx->buf("kg_e", (size_t)KL * N * 8);
    int8_t *de = (int8_t *)ctx->buf("kg_es", N);
    std::vector<u64> ha((size_t)KL * N);
    std::vector<int8_t> he(N);
    const std::vector<int> all = iota(KL);
    kern::LimbSet As{A, KL, KL, 1, all}, Bs{Bv, KL, KL, 1, all}, Es{Er, KL, KL, 1, all};
    for (size_t ki = 0; ki < am.size(); ki++) {
        const uint32_t g = gal[ki];
        const bool rl = am[ki] == FG_RELIN;
        if (rl) kern::pointwise(ctx, S, S, Sg, KL, all);   // s^2 (NTT domain)
        else kern::automorphism(ctx, S, Sg, KL, g);        // phi_g(s)
        for (int j = 0; j < beta; j++) {
            const u64 idx = ((u64)(rl ? 0 : g) << 8) | (u64)j;
            hm::sample_uniform(seed, 2, idx, ctx->primes.data(), KL, N, ha.data());
            hm::sample_gauss(seed, 3, idx, N, he.data());
            CUDA_TRY(cudaMemcpyAsync(A, ha.data(), ha.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
            CUDA_TRY(cudaMemcpyAsync(de, he.data(), N, cudaMemcpyHostToDevice, ctx->stream));
            kern::ntt_fwd(ctx, As, As);
            kern::pointwise(ctx, A, S, Bv, KL, all);
            kern::neg(ctx, Bv, Bv, KL, all);
            kern::small_to_res(ctx, de, Er, KL, g_pidx_all[ctx]);
            kern::ntt_fwd(ctx, Es, Es);
            kern::add(ctx, Bv, Er, Bv, KL, all);
            const int d0 = j * ctx->alpha, dn = std::min(ctx->alpha, L + 1 - d0);
            kern::scalar(ctx, Sg + (size_t)d0 * N, T, dn, iota(dn, d0), g_pmodq[ctx] + 2 * d0);
            kern::add(ctx, Bv + (size_t)d0 * N, T, Bv + (size_t)d0 * N, dn, iota(dn, d0));
            kern::ntt_inv(ctx, Bs, Bs);
            u64 *dst = (u64 *)(ew.b.data() + data_off) + ki * key_w + ((size_t)j * 2) * KL * limb_w;
            CUDA_TRY(cudaMemcpyAsync(dst, Bv, (size_t)KL * N * 8, cudaMemcpyDeviceToHost, ctx->stream));
            sync(ctx);
            memcpy(dst + (size_t)KL * N, ha.data(), ha.size() * 8);
        }
    }
    const u64 sum = checksum(ew.b.data(), ew.b.size() - 8);
    memcpy(ew.b.data() + ew.b.size() - 8, &sum, 8);
    *sk_blob = blob_copy(sw.b);
    *sk_len = sw.b.size();
    *evk_blob = blob_copy(ew.b);
    *evk_len = ew.b.size();
    API_CATCH(ctx)
}

int fg_encode_plain(fg_ctx *ctx, const double *slots, int n_slots, double scale, int level,
                    uint64_t *out)
{
    if (!ctx) return FG_EINVAL;
    API_TRY
    FG_CHECK(level >= 0 && level < ctx->nq && (slots || n_slots == 0) && out, FG_EINVAL,
             "bad encode arguments");
    FG_CHECK(scale > 0 && std::isfinite(scale), FG_EINVAL, "bad scale");
    std::vector<u64> h((size_t)(level + 1) * ctx->n);
    hm::encode(ctx->log_n, slots, n_slots, scale, ctx->primes.data(), level + 1, h.data());
    if (is_device_ptr(out)) {
        CUDA_TRY(cudaMemcpyAsync(out, h.data(), h.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
        sync(ctx);
    } else {
        memcpy(out, h.data(), h.size() * 8);
    }
    API_CATCH(ctx)
}

int fg_encrypt(fg_ctx *ctx, const void *sk_blob, size_t sk_len, uint64_t seed, uint64_t index,
               const uint64_t *pt, int level, uint64_t *out)
{
    if (!ctx) return FG_EINVAL;
    API_TRY
    FG_CHECK(level >= 0 && level < ctx->nq, FG_ELEVEL, "level out of range");
    const int N = ctx->n, nl = level + 1;
    const u64 *S = secret_ntt(ctx, sk_blob, sk_len);
    const u64 *dpt = stage_in(ctx, pt, (size_t)nl * N, "io_pt");
    std::vector<u64> ha((size_t)nl * N);
    std::vector<int8_t> he(N);
    hm::sample_uniform(seed, 4, index, ctx->primes.data(), nl, N, ha.data());
    hm::sample_gauss(seed, 5, index, N, he.data());
    u64 *dout = is_device_ptr(out) ? out : (u64 *)ctx->buf("io_ct", (size_t)2 * nl * N * 8);
    encrypt_dev(ctx, S, seed, index, dpt, level, dout, ha.data(), he.data());
    stage_out(ctx, out, dout, (size_t)2 * nl * N);
    sync(ctx);
    API_CATCH(ctx)
}

// Packing and encryption of the features (seeded: the uniform part drawn
// by sample_uniform_wide and only c0 written, [nb][L+1][N]; otherwise full
// ciphertexts [nb][2][L+1][N]).
static void pack_features_impl(fg_ctx *ctx, const void *sk_blob, size_t sk_len, uint64_t seed,
                               const double *X, int V, int F, const int32_t *perm, int t,
                               uint64_t *out_cts, int *n_out, bool seeded)
{
    const int N = ctx->n, M = ctx->slots, L = ctx->L(), nl = L + 1;
    FG_CHECK(X && perm && out_cts && V >= 1 && F >= 1, FG_EINVAL, "bad packing arguments");
    FG_CHECK(t >= 1 && (t & (t - 1)) == 0 && t <= M, FG_EINVAL, "t must be a power of two");
    const int B = M / t, nb = (F + t - 1) / t;
    FG_CHECK(V <= B, FG_EINVAL, "nodes do not fit a block");
    for (int v = 0; v < V; v++) FG_CHECK(perm[v] >= 0 && perm[v] < B, FG_EINVAL, "perm out of range");
    const u64 *S = secret_ntt(ctx, sk_blob, sk_len);
    const bool dev_out = is_device_ptr(out_cts) && !seeded;
    const size_t ct_w = (size_t)2 * nl * N, out_w = seeded ? (size_t)nl * N : ct_w;
    const int chunk = 16;
    std::vector<std::vector<u64>> pts(chunk, std::vector<u64>((size_t)nl * N));
    std::vector<std::vector<u64>> as(chunk, std::vector<u64>((size_t)nl * N));
    std::vector<std::vector<int8_t>> es(chunk, std::vector<int8_t>(N));
    u64 *dpt = (u64 *)ctx->buf("pack_pt", (size_t)nl * N * 8);
    u64 *dct = dev_out ? nullptr : (u64 *)ctx->buf("pack_ct", ct_w * 8);
    for (int b0 = 0; b0 < nb; b0 += chunk) {
        const int cn = std::min(chunk, nb - b0);
        int bad = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : bad)
        for (int c = 0; c < cn; c++) {
            const int b = b0 + c;
            std::vector<double> z(M, 0.0);
            for (int k = 0; k < t; k++) {
                const int f = b * t + k;
                if (f >= F) continue;
                for (int v = 0; v < V; v++) z[(size_t)k * B + perm[v]] = X[(size_t)v * F + f];
            }
            try {
                hm::encode(ctx->log_n, z.data(), M, ctx->scale, ctx->primes.data(), nl, pts[c].data());
            } catch (...) {
                bad = 1;
            }
            if (seeded)
                hm::sample_uniform_wide(seed, hm::kSeededPurpose, (u64)b, ctx->primes.data(), nl, N,
                                        as[c].data());
            else
                hm::sample_uniform(seed, 4, (u64)b, ctx->primes.data(), nl, N, as[c].data());
            hm::sample_gauss(seed, 5, (u64)b, N, es[c].data());
        }
        FG_CHECK(!bad, FG_EINVAL, "feature value cannot be encoded");
        for (int c = 0; c < cn; c++) {
            const int b = b0 + c;
            CUDA_TRY(cudaMemcpyAsync(dpt, pts[c].data(), (size_t)nl * N * 8, cudaMemcpyHostToDevice,
                                     ctx->stream));
            u64 *o = dev_out ? out_cts + (size_t)b * ct_w : dct;
            encrypt_dev(ctx, S, seed, (u64)b, dpt, L, o, as[c].data(), es[c].data());
            if (!dev_out) {   // seeded: c0 only
                CUDA_TRY(cudaMemcpyAsync(out_cts + (size_t)b * out_w, dct, out_w * 8, cudaMemcpyDefault,
                                         ctx->stream));
                sync(ctx);
            }
        }
    }
    if (n_out) *n_out = nb;
    sync(ctx);
}

int fg_pack_features(fg_ctx *ctx, const void *sk_blob, size_t sk_len, uint64_t seed,
                     const double *X, int V, int F, const int32_t *perm, int t, uint64_t *out_cts,
                     int *n_out)
{
    if (!ctx) return FG_EINVAL;
    API_TRY
    pack_features_impl(ctx, sk_blob, sk_len, seed, X, V, F, perm, t, out_cts, n_out, false);
    API_CATCH(ctx)
}

int fg_pack_features_seeded(fg_ctx *ctx, const void *sk_blob, size_t sk_len, uint64_t seed,
                            const double *X, int V, int F, const int32_t *perm, int t, uint64_t *out_c0,
                            int *n_out)
{
    if (!ctx) return FG_EINVAL;
    API_TRY
    pack_features_impl(ctx, sk_blob, sk_len, seed, X, V, F, perm, t, out_c0, n_out, true);
    API_CATCH(ctx)
}

int fg_expand_seeded(fg_ctx *ctx, uint64_t seed, const uint64_t *c0, int n, int level, uint64_t *out_cts)
{
    if (!ctx) return FG_EINVAL;
    API_TRY
    FG_CHECK(c0 && out_cts && n >= 0 && n <= 65535 && level >= 0 && level < ctx->nq, FG_EINVAL,
             "bad seeded-ciphertext arguments");
    const int N = ctx->n, nl = level + 1;
    const size_t c0_w = (size_t)nl * N, ct_w = 2 * c0_w;
    const bool dev_out = is_device_ptr(out_cts);
    u64 *d = dev_out ? out_cts : (u64 *)ctx->buf("expand_ct", (size_t)n * ct_w * 8);
    if (n) {
        const u64 *dc0 = c0;
        if (!is_device_ptr(c0)) {
            u64 *s = (u64 *)ctx->buf("expand_c0", (size_t)n * c0_w * 8);
            CUDA_TRY(cudaMemcpyAsync(s, c0, (size_t)n * c0_w * 8, cudaMemcpyHostToDevice, ctx->stream));
            dc0 = s;
        }
        kern::expand_uniform(ctx, ctx->stream, d, ct_w, dc0, n, nl, seed, 0);
        if (!dev_out)
            CUDA_TRY(cudaMemcpyAsync(out_cts, d, (size_t)n * ct_w * 8, cudaMemcpyDeviceToHost, ctx->stream));
    }
    sync(ctx);
    API_CATCH(ctx)
}

int fg_pack_neighbor_copies(fg_ctx *ctx, const void *sk_blob, size_t sk_len, uint64_t seed,
                            const double *X, int V, int F, const int32_t *nbr, int n, const int32_t *perm,
                            uint64_t *out_cts)
{
    if (!ctx) return FG_EINVAL;
    API_TRY
    FG_CHECK(X && nbr && perm && out_cts && V >= 1 && F >= 1 && n >= 1, FG_EINVAL,
             "bad neighbour-copy arguments");
    for (size_t e = 0; e < (size_t)V * n; e++)
        FG_CHECK(nbr[e] >= -1 && nbr[e] < V, FG_EINVAL, "neighbour index out of range");
    const size_t ct_w = (size_t)2 * ctx->nq * ctx->n;
    std::vector<double> Xk((size_t)V * F);
    for (int k = 0; k < n; k++) {
        for (int v = 0; v < V; v++) {
            const int u = nbr[(size_t)v * n + k];
            for (int f = 0; f < F; f++) Xk[(size_t)v * F + f] = u >= 0 ? X[(size_t)u * F + f] : 0.0;
        }
        const int rc = fg_pack_features(ctx, sk_blob, sk_len, seed + (uint64_t)k, Xk.data(), V, F, perm, 1,
                                        out_cts + (size_t)k * F * ct_w, nullptr);
        if (rc != FG_OK) return rc;
    }
    API_CATCH(ctx)
}

int fg_decrypt(fg_ctx *ctx, const void *sk_blob, size_t sk_len, const uint64_t *ct, int level,
               uint64_t *out_pt)
{
    if (!ctx) return FG_EINVAL;
    API_TRY
    FG_CHECK(level >= 0 && level < ctx->nq, FG_ELEVEL, "level out of range");
    const int N = ctx->n, nl = level + 1;
    const u64 *S = secret_ntt(ctx, sk_blob, sk_len);
    const u64 *dct = stage_in(ctx, ct, (size_t)2 * nl * N, "io_ct");
    u64 *m = is_device_ptr(out_pt) ? out_pt : (u64 *)ctx->buf("io_pt_out", (size_t)nl * N * 8);
    decrypt_dev(ctx, S, dct, level, m);
    stage_out(ctx, out_pt, m, (size_t)nl * N);
    sync(ctx);
    API_CATCH(ctx)
}

int fg_decrypt_decode(fg_ctx *ctx, const void *sk_blob, size_t sk_len, const uint64_t *ct,
                      int level, double scale, double *out_slots)
{
    if (!ctx) return FG_EINVAL;
    API_TRY
    FG_CHECK(level >= 0 && level < ctx->nq && out_slots && scale > 0, FG_EINVAL, "bad arguments");
    const int N = ctx->n, nl = level + 1;
    const u64 *S = secret_ntt(ctx, sk_blob, sk_len);
    const u64 *dct = stage_in(ctx, ct, (size_t)2 * nl * N, "io_ct");
    u64 *m = (u64 *)ctx->buf("io_pt_out", (size_t)nl * N * 8);
    decrypt_dev(ctx, S, dct, level, m);
    const int use = std::min(nl, 2);
    std::vector<u64> h((size_t)use * N);
    CUDA_TRY(cudaMemcpyAsync(h.data(), m, h.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    sync(ctx);
    std::vector<double> coef(N);
    const u64 q0 = ctx->primes[0];
    if (use == 1) {
        for (int i = 0; i < N; i++) {
            const u64 r = h[i];
            const double c = r > q0 / 2 ? -(double)(q0 - r) : (double)r;
            coef[i] = c / scale;
        }
    } else {
        const u64 q1 = ctx->primes[1];
        const u64 inv = hm::invmod(q0 % q1, q1);
        const u128 Q = (u128)q0 * q1;
        for (int i = 0; i < N; i++) {
            const u64 r0 = h[i], r1 = h[(size_t)N + i];
            const u64 d = hm::mulmod((r1 + q1 - r0 % q1) % q1, inv, q1);
            const u128 x = (u128)r0 + (u128)q0 * d;
            const double c = x > Q / 2 ? -(double)(Q - x) : (double)x;
            coef[i] = c / scale;
        }
    }
    hm::decode(ctx->log_n, coef.data(), out_slots);
    API_CATCH(ctx)
}

// ---------------------------------------------------------------- server side
int fg_load_evk(fg_ctx *ctx, const void *evk_blob, size_t len, fg_keys **out)
{
    if (!ctx) return FG_EINVAL;
    fg_keys *keys = nullptr;
    API_TRY
    FG_CHECK(evk_blob && out, FG_EINVAL, "null argument");
    *out = nullptr;
    const uint8_t *p = (const uint8_t *)evk_blob;
    FG_CHECK(len >= 8 + 6 * 4 + 8 && memcmp(p, kEvkMagic, 8) == 0, FG_EKEY, "not an evk blob");
    u64 sum;
    memcpy(&sum, p + len - 8, 8);
    FG_CHECK(checksum(p, len - 8) == sum, FG_EKEY, "evk checksum mismatch");
    Reader r{p, len - 8};
    r.off = 8;
    FG_CHECK(r.get<uint32_t>() == 1, FG_EKEY, "evk version");
    const uint32_t log_n = r.get<uint32_t>(), nq = r.get<uint32_t>(), np = r.get<uint32_t>(),
                   alpha = r.get<uint32_t>(), nk = r.get<uint32_t>();
    FG_CHECK((int)log_n == ctx->log_n && (int)nq == ctx->nq && (int)np == ctx->np &&
                 (int)alpha == ctx->alpha, FG_EKEY, "evk made for other parameters");
    for (int i = 0; i < ctx->nq + ctx->np; i++)
        FG_CHECK(r.get<u64>() == ctx->primes[i], FG_EKEY, "evk made for other primes");
    const int N = ctx->n, KL = ctx->nq + ctx->np, beta = ctx->n_digits(ctx->L());
    const size_t key_w = (size_t)beta * 2 * KL * N;
    std::vector<std::pair<int32_t, uint32_t>> ids(nk);
    for (uint32_t i = 0; i < nk; i++) {
        ids[i].first = r.get<int32_t>();
        ids[i].second = r.get<uint32_t>();
        FG_CHECK((ids[i].first == FG_RELIN && ids[i].second == 1u) ||
                     (ids[i].first > 0 && ids[i].first < ctx->slots &&
                      ids[i].second == (uint32_t)hm::powmod(5, ids[i].first, 2 * (u64)N)),
                 FG_EKEY, "evk key entry inconsistent");
    }
    FG_CHECK(r.off + nk * key_w * 8 == r.len, FG_EKEY, "evk size mismatch");
    keys = new fg_keys;
    keys->ctx = ctx;
    const u64 *data = (const u64 *)(p + r.off);
    const std::vector<int> all = iota(KL);
    for (uint32_t i = 0; i < nk; i++) {
        KeyDev kd;
        kd.amount = ids[i].first;
        kd.galois = ids[i].second;
        CUDA_TRY(cudaMalloc(&kd.d, key_w * 8));
        keys->keys[kd.amount] = kd;
        CUDA_TRY(cudaMemcpyAsync(kd.d, data + i * key_w, key_w * 8, cudaMemcpyHostToDevice, ctx->stream));
        kern::LimbSet ks{kd.d, KL, KL, 2 * beta, all};
        kern::ntt_fwd(ctx, ks, ks);
        kern::to_mont(ctx, kd.d, 2 * beta * KL, all);
    }
    sync(ctx);
    *out = keys;
    keys = nullptr;
    }
    catch (const fg_error &e) {
        if (keys) fg_keys_destroy(keys);
        ctx->err = e.what();
        return e.code;
    }
    catch (const std::exception &e) {
        if (keys) fg_keys_destroy(keys);
        ctx->err = e.what();
        return FG_EOOM;
    }
    return FG_OK;
}

int fg_keys_destroy(fg_keys *keys)
{
    if (!keys) return FG_OK;
    if (keys->ctx) cudaStreamSynchronize(keys->ctx->stream);
    for (auto &kv : keys->keys) cudaFree(kv.second.d);
    delete keys;
    return FG_OK;
}

int fg_keys_export(const fg_keys *keys, int32_t amount, int digit, uint64_t *b_out, uint64_t *a_out)
{
    if (!keys || !keys->ctx) return FG_EINVAL;
    fg_ctx *ctx = keys->ctx;
    API_TRY
    const int N = ctx->n, KL = ctx->nq + ctx->np, beta = ctx->n_digits(ctx->L());
    FG_CHECK(digit >= 0 && digit < beta && b_out && a_out, FG_EINVAL, "bad digit");
    const KeyDev &k = keys->get(amount == FG_RELIN ? FG_RELIN
                                                   : ((amount % ctx->slots) + ctx->slots) % ctx->slots);
    u64 *t = (u64 *)ctx->buf("kx", (size_t)2 * KL * N * 8);
    CUDA_TRY(cudaMemcpyAsync(t, k.d + (size_t)digit * 2 * KL * N, (size_t)2 * KL * N * 8,
                             cudaMemcpyDeviceToDevice, ctx->stream));
    const std::vector<int> all = iota(KL);
    kern::from_mont(ctx, t, 2 * KL, all);
    kern::LimbSet ts{t, KL, KL, 2, all};
    kern::ntt_inv(ctx, ts, ts);
    stage_out(ctx, b_out, t, (size_t)KL * N);
    stage_out(ctx, a_out, t + (size_t)KL * N, (size_t)KL * N);
    sync(ctx);
    API_CATCH(ctx)
}

// ---------------------------------------------------------------- single ops
int fg_poly_mul(fg_ctx *ctx, const uint64_t *a, const uint64_t *b, int level, uint64_t *c)
{
    if (!ctx) return FG_EINVAL;
    API_TRY
    FG_CHECK(level >= 0 && level < ctx->nq, FG_ELEVEL, "level out of range");
    const int N = ctx->n, nl = level + 1;
    const std::vector<int> pid = iota(nl);
    const u64 *da = stage_in(ctx, a, (size_t)nl * N, "pm_a");
    const u64 *db = stage_in(ctx, b, (size_t)nl * N, "pm_b");
    u64 *ta = (u64 *)ctx->buf("pm_ta", (size_t)nl * N * 8);
    u64 *tb = (u64 *)ctx->buf("pm_tb", (size_t)nl * N * 8);
    kern::LimbSet sa{const_cast<u64 *>(da), nl, nl, 1, pid}, sb{const_cast<u64 *>(db), nl, nl, 1, pid};
    kern::LimbSet ta_s{ta, nl, nl, 1, pid}, tb_s{tb, nl, nl, 1, pid};
    kern::ntt_fwd(ctx, sa, ta_s);
    kern::ntt_fwd(ctx, sb, tb_s);
    kern::pointwise(ctx, ta, tb, ta, nl, pid);
    kern::ntt_inv(ctx, ta_s, ta_s);
    stage_out(ctx, c, ta, (size_t)nl * N);
    sync(ctx);
    API_CATCH(ctx)
}

int fg_ntt(fg_ctx *ctx, uint64_t *data, int count, const int *prime_idx, int period, int inverse)
{
    if (!ctx) return FG_EINVAL;
    API_TRY
    FG_CHECK(data && prime_idx && period >= 1 && count >= 0 && count % period == 0, FG_EINVAL,
             "bad ntt arguments");
    FG_CHECK(is_device_ptr(data), FG_EINVAL, "fg_ntt works on device memory");
    std::vector<int> pid(prime_idx, prime_idx + period);
    for (int p : pid) FG_CHECK(p >= 0 && p < ctx->nq + ctx->np, FG_EINVAL, "bad prime index");
    kern::LimbSet s{data, period, period, count / period, pid};
    if (inverse) kern::ntt_inv(ctx, s, s);
    else kern::ntt_fwd(ctx, s, s);
    sync(ctx);
    API_CATCH(ctx)
}

int fg_rescale(fg_ctx *ctx, const uint64_t *ct, int level, uint64_t *out)
{
    if (!ctx) return FG_EINVAL;
    API_TRY
    FG_CHECK(level >= 1 && level < ctx->nq, FG_ELEVEL, "rescale needs 1 <= level <= L");
    const int N = ctx->n;
    const u64 *d = stage_in(ctx, ct, (size_t)2 * (level + 1) * N, "io_ct");
    u64 *o = is_device_ptr(out) ? out : (u64 *)ctx->buf("io_rs", (size_t)2 * level * N * 8);
    FG_CHECK(o != d, FG_EINVAL, "rescale output must not alias its input");
    kern::rescale_coef(ctx, d, level + 1, o, level, 2, level);
    stage_out(ctx, out, o, (size_t)2 * level * N);
    sync(ctx);
    API_CATCH(ctx)
}

int fg_mul_relin_rescale(fg_ctx *ctx, const fg_keys *keys, const uint64_t *a, const uint64_t *b,
                         int n, int level, uint64_t *out)
{
    if (!ctx || !keys) return FG_EINVAL;
    API_TRY
    FG_CHECK(a && b && out && n >= 1, FG_EINVAL, "null argument");
    FG_CHECK(level >= 1 && level < ctx->nq, FG_ELEVEL, "CMult needs a level >= 1");
    const KeyDev &rk = keys->get(FG_RELIN);
    const int N = ctx->n, nl = level + 1, E = ctx->ext(level), beta = ctx->n_digits(level);
    const size_t w = (size_t)n * 2 * nl * N, pw = (size_t)nl * N;
    const u64 *da = stage_in(ctx, a, w, "mul_a");
    const u64 *db = b == a ? da : stage_in(ctx, b, w, "mul_b");
    const std::vector<int> pid = iota(nl);
    u64 *A = (u64 *)ctx->buf("mul_an", w * 8);
    kern::LimbSet as{const_cast<u64 *>(da), nl, nl, 2 * n, pid}, an{A, nl, nl, 2 * n, pid};
    kern::ntt_fwd(ctx, as, an);
    u64 *B = A;
    if (b != a) {
        B = (u64 *)ctx->buf("mul_bn", w * 8);
        kern::LimbSet bs{const_cast<u64 *>(db), nl, nl, 2 * n, pid}, bn{B, nl, nl, 2 * n, pid};
        kern::ntt_fwd(ctx, bs, bn);
    }
    // lane (d0, d2) per pair, d1 aside (NTT domain)
    u64 *Ln = (u64 *)ctx->buf("mul_lane", w * 8);
    u64 *D1 = (u64 *)ctx->buf("mul_d1", (size_t)n * pw * 8);
    u64 *T = (u64 *)ctx->buf("mul_t", (size_t)n * pw * 8);
    for (int c = 0; c < n; c++) {
        const u64 *a0 = A + (size_t)c * 2 * pw, *a1 = a0 + pw;
        const u64 *b0 = B + (size_t)c * 2 * pw, *b1 = b0 + pw;
        u64 *l0 = Ln + (size_t)c * 2 * pw;
        kern::pointwise(ctx, a0, b0, l0, nl, pid);
        kern::pointwise(ctx, a1, b1, l0 + pw, nl, pid);
        kern::pointwise(ctx, a0, b1, D1 + (size_t)c * pw, nl, pid);
        kern::pointwise(ctx, a1, b0, T + (size_t)c * pw, nl, pid);
    }
    kern::add(ctx, D1, T, D1, n * nl, pid);
    // u = KS(d2) + P d0 (part 0), then + P d1 (part 1): ModDown gives
    // (d0, d1) + KS(d2) exactly, and the rescale is fused into it
    u64 *digits = (u64 *)ctx->buf("mul_digits", (size_t)n * beta * E * N * 8);
    kern::modup(ctx, Ln, nl, n, level, digits);
    u64 *u = (u64 *)ctx->buf("mul_u", (size_t)n * 2 * E * N * 8);
    kern::ks_multi(ctx, {&rk}, {u}, Ln, nl, n, level, digits);
    kern::scalar(ctx, D1, T, n * nl, pid, ctx->d_pmodq);
    for (int c = 0; c < n; c++) {
        u64 *u1 = u + ((size_t)c * 2 + 1) * E * N;
        kern::add(ctx, u1, T + (size_t)c * pw, u1, nl, pid);
    }
    u64 *R = (u64 *)ctx->buf("mul_r", w * 8);
    kern::moddown_rescale_to_lane(ctx, u, n, level, R, nl);
    std::vector<int> top(nl, -1);
    for (int i = 0; i < level; i++) top[i] = i;
    kern::LimbSet rs{R, nl, nl, 2 * n, top};
    kern::ntt_inv(ctx, rs, rs);
    const size_t ow = (size_t)n * 2 * level * N;
    u64 *O = is_device_ptr(out) ? out : (u64 *)ctx->buf("mul_o", ow * 8);
    kern::copy_limbs(ctx, R, nl, O, level, 2 * n, level);
    if (O != out) stage_out(ctx, out, O, ow);
    sync(ctx);
    API_CATCH(ctx)
}

int fg_rotate(fg_ctx *ctx, const fg_keys *keys, const uint64_t *ct, int level, int k, uint64_t *out)
{
    if (!ctx || !keys) return FG_EINVAL;
    API_TRY
    FG_CHECK(level >= 0 && level < ctx->nq, FG_ELEVEL, "level out of range");
    const int N = ctx->n, nl = level + 1, M = ctx->slots;
    const int km = ((k % M) + M) % M;
    const u64 *d = stage_in(ctx, ct, (size_t)2 * nl * N, "io_ct");
    u64 *lane = (u64 *)ctx->buf("rot_lane", (size_t)2 * nl * N * 8);
    u64 *res = (u64 *)ctx->buf("rot_out", (size_t)2 * nl * N * 8);
    const std::vector<int> pid = iota(nl);
    kern::LimbSet src{const_cast<u64 *>(d), nl, nl, 2, pid}, ls{lane, nl, nl, 2, pid};
    if (km == 0) {
        stage_out(ctx, out, d, (size_t)2 * nl * N);
        sync(ctx);
        return FG_OK;
    }
    const KeyDev &key = keys->get(km);
    kern::ntt_fwd(ctx, src, ls);
    u64 *digits = (u64 *)ctx->buf("rot_digits",
                                  (size_t)ctx->n_digits(level) * ctx->ext(level) * N * 8);
    kern::modup(ctx, lane, nl, 1, level, digits);
    kern::rotate_mac(ctx, key, lane, nl, 1, level, digits, {{res, nullptr}}, nl);
    kern::LimbSet rs{res, nl, nl, 2, pid};
    kern::ntt_inv(ctx, rs, rs);
    stage_out(ctx, out, res, (size_t)2 * nl * N);
    sync(ctx);
    API_CATCH(ctx)
}

}  // extern "C"
