// layer.cu -- plans on the device and the encrypted layer A-hat X W.
//
// Execution of a plan (paper Sec. 3.2-3.3; the plan itself is planner.cpp):
//   1. combination: t = 1: integer constants times each packed input,
//      summed in the coefficient domain (one pass over X for all output
//      columns), one rescale, then the column ciphertexts go to the NTT
//      domain; t > 1: NTT of the inputs, block-replicated W masks,
//      rescale, log t rotate-and-sum steps;
//   2. SpIntra-CA groups: per input lane one ModUp of c1 (hoisted, shared by
//      all its rotation amounts), per rotation one key-switching inner
//      product and ModDown whose epilogue multiplies the rotated ciphertext
//      by every mask that uses it and adds it into the output lanes and the
//      accumulator; kept values (rotation 0) are masked the same way; then
//      every output and the group's accumulator are rescaled and the running
//      accumulator, dropped one limb, receives the group's arrivals;
//   3. the accumulator returns to the coefficient domain.
// All F' output columns share the plan, so every kernel runs over all
// columns at once and each rotation key is read once per rotation.
#include <omp.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "fg_internal.h"
#include "modarith.cuh"

namespace {

bool is_dev(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool is_pinned(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

std::vector<int> iota(int n, int start = 0)
{
    std::vector<int> v(n);
    for (int i = 0; i < n; i++) v[i] = start + i;
    return v;
}

// put one encoded mask of the plan on the device over q_0..q_level and the
// special primes (the latter lifted from limb 0: every mask coefficient is
// below q_0 / 2 in magnitude), NTT domain, Montgomery form: [E][N]
void upload_mask(fg_ctx *ctx, MaskC &m, const u64 *coeffs_host_or_dev)
{
    const int N = ctx->n, nl = m.level + 1, E = ctx->ext(m.level);
    if (!m.d) CUDA_TRY(cudaMalloc(&m.d, (size_t)E * N * 8));
    CUDA_TRY(cudaMemcpyAsync(m.d, coeffs_host_or_dev, (size_t)nl * N * 8, cudaMemcpyDefault,
                             ctx->stream));
    kern::lift_special(ctx, m.d, m.d + (size_t)nl * N);
    std::vector<int> pid(E);
    for (int i = 0; i < E; i++) pid[i] = ctx->ext_prime(m.level, i);
    kern::LimbSet s{m.d, E, E, 1, pid};
    kern::ntt_fwd(ctx, s, s);
    kern::to_mont(ctx, m.d, E, pid);
}

void encode_mask(const fg_ctx *ctx, const MaskC &m, u64 *out)
{
    std::vector<double> z(ctx->slots, 0.0);
    for (size_t i = 0; i < m.slots.size(); i++) z[m.slots[i]] = m.values[i];
    hm::encode(ctx->log_n, z.data(), ctx->slots, (double)ctx->primes[m.level], ctx->primes.data(),
               m.level + 1, out);
}

}  // namespace

extern "C" {

}  // extern "C"

// masks encoded on the host (all cores), uploaded, NTT, Montgomery form;
// the combination constants in Montgomery form for every limb
static void finish_plan(fg_ctx *ctx, fg_plan *pl, bool no_encode)
{
    const int N = ctx->n, F = pl->F, Fp = pl->Fp;
    const int nm = (int)pl->masks.size();
    if (no_encode) {   // timing-only plan: zero masks, no host encoding
        for (MaskC &m : pl->masks) {
            const size_t bytes = (size_t)ctx->ext(m.level) * N * 8;
            CUDA_TRY(cudaMalloc(&m.d, bytes));
            CUDA_TRY(cudaMemsetAsync(m.d, 0, bytes, ctx->stream));
        }
    }
    const int chunk = 32;
    std::vector<std::vector<u64>> enc(chunk);
    for (int m0 = 0; m0 < (no_encode ? 0 : nm); m0 += chunk) {
        const int cn = std::min(chunk, nm - m0);
        int bad = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : bad)
        for (int c = 0; c < cn; c++) {
            const MaskC &m = pl->masks[m0 + c];
            enc[c].resize((size_t)(m.level + 1) * N);
            try {
                encode_mask(ctx, m, enc[c].data());
            } catch (...) {
                bad = 1;
            }
        }
        FG_CHECK(!bad, FG_EINVAL, "mask cannot be encoded");
        for (int c = 0; c < cn; c++) upload_mask(ctx, pl->masks[m0 + c], enc[c].data());
        CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    }
    if (pl->t == 1) {
        const int l0 = pl->in_level, nl = l0 + 1;
        std::vector<u64> h((size_t)nl * F * Fp);
        for (int i = 0; i < nl; i++) {
            const u64 q = ctx->primes[i];
            for (size_t e = 0; e < (size_t)F * Fp; e++) {
                const i64 c = pl->comb_consts[e];
                const u64 r = c >= 0 ? (u64)c % q : (q - ((u64)(-(c + 1)) % q + 1) % q) % q;
                h[(size_t)i * F * Fp + e] = hm::to_mont(r, q);
            }
        }
        CUDA_TRY(cudaMalloc(&pl->d_comb, h.size() * 8));
        CUDA_TRY(cudaMemcpy(pl->d_comb, h.data(), h.size() * 8, cudaMemcpyHostToDevice));
    }
}

extern "C" {

int fg_plan_build(fg_ctx *ctx, const int32_t *row_ptr, const int32_t *col, const double *val,
                  int V, const double *W, int F, int Fp, const int32_t *perm,
                  const fg_plan_opts *opts, fg_plan **out)
{
    if (!ctx) return FG_EINVAL;
    fg_plan *pl = nullptr;
    try {
        FG_CHECK(row_ptr && (col || V == 0) && W && perm && out, FG_EINVAL, "null argument");
        *out = nullptr;
        fg_plan_opts o{0, 0, 1, 0, 0, 0, 0};
        if (opts) o = *opts;
        pl = new fg_plan;
        pl->ctx = ctx;
        planner::build(*pl, *ctx, row_ptr, col, val, V, W, F, Fp, perm, o);
        finish_plan(ctx, pl, o.no_encode != 0);
        *out = pl;
        return FG_OK;
    } catch (const fg_error &e) {
        ctx->err = e.what();
        fg_plan_destroy(pl);
        return e.code;
    } catch (const std::exception &e) {
        ctx->err = e.what();
        fg_plan_destroy(pl);
        return FG_EOOM;
    }
}

int fg_plan_build_inter(fg_ctx *ctx, const int32_t *nbr, const double *wts, int V, int n,
                        const double *W, int F, int Fp, const int32_t *perm,
                        const fg_plan_opts *opts, fg_plan **out)
{
    if (!ctx) return FG_EINVAL;
    fg_plan *pl = nullptr;
    try {
        FG_CHECK(nbr && wts && W && perm && out, FG_EINVAL, "null argument");
        *out = nullptr;
        fg_plan_opts o{0, 0, 1, 0, 0, 0, 0};
        if (opts) o = *opts;
        pl = new fg_plan;
        pl->ctx = ctx;
        planner::build_inter(*pl, *ctx, nbr, wts, V, n, W, F, Fp, perm, o);
        finish_plan(ctx, pl, o.no_encode != 0);
        *out = pl;
        return FG_OK;
    } catch (const fg_error &e) {
        ctx->err = e.what();
        fg_plan_destroy(pl);
        return e.code;
    } catch (const std::exception &e) {
        ctx->err = e.what();
        fg_plan_destroy(pl);
        return FG_EOOM;
    }
}

int fg_plan_destroy(fg_plan *plan)
{
    if (!plan) return FG_OK;
    if (plan->ctx) cudaStreamSynchronize(plan->ctx->stream);
    for (auto &m : plan->masks) cudaFree(m.d);
    cudaFree(plan->d_comb);
    delete plan;
    return FG_OK;
}

int fg_plan_info(const fg_plan *pl, fg_plan_info_t *info)
{
    if (!pl || !info) return FG_EINVAL;
    memset(info, 0, sizeof(*info));
    info->t = pl->t;
    info->B = pl->B;
    info->n_in = pl->n_copies ? pl->n_copies * pl->F : pl->t == 1 ? pl->F : (pl->F + pl->t - 1) / pl->t;
    info->n_out = pl->Fp;
    info->in_level = pl->in_level;
    info->out_level = pl->out_level;
    info->n_groups = (int)pl->groups.size();
    info->n_masks = (int)pl->masks.size();
    int32_t tmp[1];
    int nk = 0;
    fg_plan_rotation_amounts(pl, tmp, 0, &nk);
    info->n_keys = nk;
    int64_t rots = (int64_t)pl->comb_rots.size(), prods = 0;
    for (auto &g : pl->groups) {
        rots += (int64_t)g.rots.size();
        prods += (int64_t)g.terms.size();
    }
    if (pl->t > 1) prods += (int64_t)pl->comb_masks.size() * pl->Fp;
    info->rotations = rots * pl->Fp;
    info->masked_products = prods * pl->Fp;
    return FG_OK;
}

int fg_plan_rotation_amounts(const fg_plan *pl, int32_t *out, int cap, int *n)
{
    if (!pl || !n) return FG_EINVAL;
    std::vector<int32_t> ks;
    for (int k : pl->comb_rots) ks.push_back(((k % pl->M) + pl->M) % pl->M);
    for (auto &g : pl->groups)
        for (auto &r : g.rots) ks.push_back(((r.second % pl->M) + pl->M) % pl->M);
    std::sort(ks.begin(), ks.end());
    ks.erase(std::unique(ks.begin(), ks.end()), ks.end());
    *n = (int)ks.size();
    if (out)
        for (int i = 0; i < std::min(cap, (int)ks.size()); i++) out[i] = ks[i];
    return (out && cap < (int)ks.size()) ? FG_EINVAL : FG_OK;
}

static std::vector<int64_t> describe_records(const fg_plan *pl)
{
    std::vector<int64_t> r = {pl->N, pl->M, pl->t, pl->B, pl->V, pl->F, pl->Fp, pl->in_level,
                              pl->out_level, pl->radix_bits, pl->aoo, (int64_t)pl->groups.size(),
                              (int64_t)pl->masks.size()};
    for (int v : pl->perm) r.push_back(v);
    if (pl->t == 1) {
        for (i64 c : pl->comb_consts) r.push_back(c);
    } else {
        for (auto &row : pl->comb_masks)
            for (int m : row) r.push_back(m);
        r.push_back((int64_t)pl->comb_rots.size());
        for (int k : pl->comb_rots) r.push_back(k);
    }
    for (auto &g : pl->groups) {
        r.insert(r.end(), {g.bit_lo, g.n_bits, g.level, g.n_in, g.n_out, (int64_t)g.rots.size()});
        for (auto &rk : g.rots) r.insert(r.end(), {rk.first, rk.second});
        r.push_back((int64_t)g.terms.size());
        for (auto &t : g.terms) r.insert(r.end(), {t.src, t.k, t.dst, t.mask});
    }
    for (auto &m : pl->masks) {
        r.push_back(m.level);
        r.push_back((int64_t)m.slots.size());
        for (size_t i = 0; i < m.slots.size(); i++) {
            int64_t bits;
            memcpy(&bits, &m.values[i], 8);
            r.push_back(m.slots[i]);
            r.push_back(bits);
        }
    }
    return r;
}

static int copy_records(const std::vector<int64_t> &r, int64_t *out, size_t cap, size_t *len)
{
    *len = r.size();
    if (!out) return FG_OK;
    if (cap < r.size()) return FG_EINVAL;
    memcpy(out, r.data(), r.size() * 8);
    return FG_OK;
}

// Records: [N, M, t, B, V, F, Fp, in_level, out_level, radix_bits, aoo,
//  n_groups, n_masks], perm[V], combination (t == 1: F*Fp constants; t > 1:
//  nb*Fp mask ids, n_rots, rots), per group [bit_lo, n_bits, level, n_in,
//  n_out, n_rots, (src, k)*, n_terms, (src, k, dst, mask)*], per mask
//  [level, nnz, (slot, value bits)*].
int fg_plan_describe(const fg_plan *pl, int64_t *out, size_t cap, size_t *len)
{
    if (!pl || !len) return FG_EINVAL;
    return copy_records(describe_records(pl), out, cap, len);
}

}  // extern "C"

// host-only planning: a context with the primes and sizes, no device tables
static void host_plan(const fg_params *prm, const int32_t *row_ptr, const int32_t *col,
                      const double *val, int V, const double *W, int F, int Fp, const int32_t *perm,
                      const fg_plan_opts *opts, fg_ctx &c, fg_plan &pl)
{
    FG_CHECK(prm->log_n >= 10 && prm->log_n <= 16 && prm->n_q >= 2 && prm->n_q <= 60 &&
                 prm->n_p >= 1 && prm->n_p <= 7 && prm->q_bits && prm->p_bits,
             FG_EINVAL, "bad parameters");
    c.log_n = prm->log_n;
    c.n = 1 << prm->log_n;
    c.slots = c.n / 2;
    c.nq = prm->n_q;
    c.np = prm->n_p;
    c.alpha = prm->alpha;
    std::vector<int> bits(prm->q_bits, prm->q_bits + prm->n_q);
    bits.insert(bits.end(), prm->p_bits, prm->p_bits + prm->n_p);
    c.primes = hm::gen_primes(c.log_n, bits);
    fg_plan_opts o{0, 0, 1, 0, 0, 0, 0};
    if (opts) o = *opts;
    planner::build(pl, c, row_ptr, col, val, V, W, F, Fp, perm, o);
}

extern "C" {

int fg_plan_dry_run(const fg_params *prm, const int32_t *row_ptr, const int32_t *col,
                    const double *val, int V, const double *W, int F, int Fp, const int32_t *perm,
                    const fg_plan_opts *opts, int64_t *out, size_t cap, size_t *len)
{
    if (!prm || !row_ptr || !W || !perm || !len) return FG_EINVAL;
    try {
        fg_ctx c;
        fg_plan pl;
        host_plan(prm, row_ptr, col, val, V, W, F, Fp, perm, opts, c, pl);
        return copy_records(describe_records(&pl), out, cap, len);
    } catch (const fg_error &e) {
        return e.code;
    } catch (const std::exception &) {
        return FG_EOOM;
    }
}

int fg_select_mode(const fg_params *prm, const int32_t *row_ptr, const int32_t *col,
                   const double *val, int V, const double *W, int F, int Fp, const int32_t *perm,
                   const fg_plan_opts *opts, int layer, int n_copies, const double lat[3],
                   double max_inter_cts, int *mode, double cost[2], int64_t counts[4])
{
    if (!prm || !row_ptr || !W || !perm || !lat || !mode || !cost) return FG_EINVAL;
    if (layer < 0 || n_copies < 1 || !(lat[0] >= 0 && lat[1] >= 0 && lat[2] >= 0)) return FG_EINVAL;
    try {
        fg_ctx c;
        fg_plan pl;
        host_plan(prm, row_ptr, col, val, V, W, F, Fp, perm, opts, c, pl);
        int64_t cnt[4];
        planner::select_mode(pl, layer, n_copies, lat, max_inter_cts, mode, cost, cnt);
        if (counts)
            for (int i = 0; i < 4; i++) counts[i] = cnt[i];
    } catch (const fg_error &e) {
        return e.code;
    } catch (const std::exception &) {
        return FG_EOOM;
    }
    return FG_OK;
}

// the learned planner's statistics of a plan (see fg_plan_features)
static void plan_features_of(const fg_plan &pl, int np, const int32_t *row_ptr, const int32_t *col,
                             int F, float *feat)
{
    const int V = pl.V, B = pl.B;
    const int32_t *perm = pl.perm.data();
    int maxdeg = 0;
    double shift_bits = 0;
    long long edges = 0;
    for (int v = 0; v < V; v++) {
        maxdeg = std::max(maxdeg, row_ptr[v + 1] - row_ptr[v]);
        for (int e = row_ptr[v]; e < row_ptr[v + 1]; e++) {
            const int u = col[e];
            if (u == v) continue;
            int d = ((perm[u] - perm[v]) % B + B) % B;
            if (d > B / 2) d -= B;
            shift_bits += 32 - __builtin_clz((unsigned)std::abs(d) | 1u);
            edges++;
        }
    }
    double rots = 0, terms = 0, ks_work = 0, mac_work = 0;
    int lanes = 1;
    for (const GroupC &g : pl.groups) {
        rots += (double)g.rots.size();
        terms += (double)g.terms.size();
        ks_work += (double)g.rots.size() * (g.level + 1 + np);
        mac_work += (double)g.terms.size() * (g.level + 1 + np);
        lanes = std::max(lanes, g.n_out);
    }
    const float f[FG_PLAN_FEATURES] = {
        (float)std::log2((double)V), (float)std::log2((double)F),
        (float)((double)row_ptr[V] / V), (float)std::log2(1.0 + maxdeg),
        (float)std::log2((double)pl.t), (float)pl.radix_bits,
        (float)(edges ? shift_bits / edges : 0.0), (float)pl.groups.size(),
        (float)std::log2(1.0 + rots), (float)std::log2(1.0 + terms), (float)lanes,
        (float)std::log2(1.0 + ks_work), (float)std::log2(1.0 + mac_work),
        (float)std::log2((double)F * (pl.in_level + 1)), (float)pl.in_level};
    for (int i = 0; i < FG_PLAN_FEATURES; i++) feat[i] = f[i];
}

int fg_plan_features(const fg_params *prm, const int32_t *row_ptr, const int32_t *col,
                     const double *val, int V, const double *W, int F, int Fp, const int32_t *perm,
                     const fg_plan_opts *opts, float *feat)
{
    if (!prm || !row_ptr || !col || !W || !perm || !feat) return FG_EINVAL;
    try {
        fg_ctx c;
        fg_plan pl;
        host_plan(prm, row_ptr, col, val, V, W, F, Fp, perm, opts, c, pl);
        plan_features_of(pl, c.np, row_ptr, col, F, feat);
    } catch (const fg_error &e) {
        return e.code;
    } catch (const std::exception &) {
        return FG_EOOM;
    }
    return FG_OK;
}

int fg_plan_features_built(const fg_plan *pl, const int32_t *row_ptr, const int32_t *col, float *feat)
{
    if (!pl || !pl->ctx || !row_ptr || !col || !feat) return FG_EINVAL;
    if (pl->n_copies) return FG_EINVAL;
    for (int v = 0; v < pl->V; v++)
        if (row_ptr[v + 1] < row_ptr[v]) return FG_EINVAL;
    for (int e = 0; e < row_ptr[pl->V]; e++)
        if (col[e] < 0 || col[e] >= pl->V) return FG_EINVAL;
    plan_features_of(*pl, pl->ctx->np, row_ptr, col, pl->F, feat);
    return FG_OK;
}

int fg_plan_set_plaintext(fg_plan *pl, int mask, const uint64_t *coeffs)
{
    if (!pl || !pl->ctx) return FG_EINVAL;
    fg_ctx *ctx = pl->ctx;
    try {
        FG_CHECK(mask >= 0 && mask < (int)pl->masks.size() && coeffs, FG_EINVAL, "bad mask index");
        upload_mask(ctx, pl->masks[mask], coeffs);
        CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    } catch (const fg_error &e) {
        ctx->err = e.what();
        return e.code;
    }
    return FG_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ the layer
// Enqueues one layer on ctx->stream with the workspace names prefixed by
// ctx->ws_prefix; waits for it only when sync is set (host buffers need it).
// seed: null for full ciphertexts [n_in][2][l0+1][N]; else in_cts holds the
// c0 parts [n_in][l0+1][N] of seeded ciphertexts 0..n_in-1 of that seed,
// whose uniform parts are regenerated on the device (kern::expand_uniform).
static void layer_exec(fg_ctx *ctx, const fg_keys *keys, const fg_plan *pl, const uint64_t *in_cts,
                       int n_in, uint64_t *out_cts, int n_out, bool sync, int *out_level,
                       const uint64_t *seed = nullptr)
{
    {
        FG_CHECK(keys && pl && in_cts && out_cts, FG_EINVAL, "null argument");
        FG_CHECK(pl->ctx == ctx && keys->ctx == ctx, FG_EINVAL, "plan or keys of another context");
        const int N = ctx->n, M = ctx->slots, Fp = pl->Fp, F = pl->F, t = pl->t;
        const int l0 = pl->in_level, nl0 = l0 + 1;
        const int nb = pl->n_copies ? pl->n_copies * F : t == 1 ? F : (F + t - 1) / t;
        FG_CHECK(n_in == nb, FG_EINVAL, "number of input ciphertexts does not match the plan");
        FG_CHECK(n_out == Fp, FG_EINVAL, "number of output ciphertexts does not match the plan");
        // every rotation key the plan needs must be present before any work
        for (int k : pl->comb_rots) keys->get(((k % M) + M) % M);
        for (auto &g : pl->groups)
            for (auto &r : g.rots) keys->get(((r.second % M) + M) % M);

        const size_t in_w = (size_t)nb * 2 * nl0 * N;
        const size_t c0_w = (size_t)nl0 * N, ct_w = 2 * c0_w;
        FG_CHECK(!seed || !pl->n_copies, FG_EINVAL, "seeded inputs: not for neighbour copies");
        const u64 *X = in_cts;
        // host inputs: staged into this workspace's buffer on its own copy
        // stream; for t = 1 in chunks of columns, the combination of each
        // chunk starting when it has arrived.  Inside a batch pass the copy
        // starts as soon as the previous layer of this workspace has read the
        // staging buffer (its combination), so it overlaps that layer's
        // aggregation and the other streams' work.
        const bool host_in = !is_dev(in_cts);
        const bool chunked = host_in && t == 1 && !pl->n_copies;
        const int kChunk = 64, n_chunks = chunked ? (F + kChunk - 1) / kChunk : 1;
        fg_ctx::CopyRes *cr = nullptr;
        u64 *c0s = nullptr;   // seeded host inputs: c0 staged contiguously, then expanded into d
        if (host_in) {
            u64 *d = (u64 *)ctx->buf("layer_in", in_w * 8);
            if (seed) c0s = (u64 *)ctx->buf("layer_in_c0", (size_t)nb * c0_w * 8);
            cr = &ctx->copies[ctx->ws_prefix];
            if (!cr->st) CUDA_TRY(cudaStreamCreateWithFlags(&cr->st, cudaStreamNonBlocking));
            if (!cr->free_ev) CUDA_TRY(cudaEventCreateWithFlags(&cr->free_ev, cudaEventDisableTiming));
            while ((int)cr->ev.size() < n_chunks + 1) {
                cudaEvent_t e;
                CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
                cr->ev.push_back(e);
            }
            if (ctx->in_batch && cr->have_free) {
                CUDA_TRY(cudaStreamWaitEvent(cr->st, cr->free_ev, 0));
            } else {   // the buffer is free once the work queued before this layer is done
                CUDA_TRY(cudaEventRecord(cr->ev[n_chunks], ctx->stream));
                CUDA_TRY(cudaStreamWaitEvent(cr->st, cr->ev[n_chunks], 0));
            }
            // columns fb .. fb + fn - 1 into the staging buffer (seeded: c0
            // only, into a buffer of its own; the compute stream, once the
            // chunk has arrived, moves it into place beside the regenerated
            // uniform parts, so that the copies run back to back)
            auto stage = [&](int fb, int fn) {
                if (seed) {   // one plain copy of the chunk's c0 (strided copies varied more)
                    CUDA_TRY(cudaMemcpyAsync(c0s + fb * c0_w, in_cts + fb * c0_w, fn * c0_w * 8,
                                             cudaMemcpyHostToDevice, cr->st));
                } else {
                    CUDA_TRY(cudaMemcpyAsync(d + fb * ct_w, in_cts + fb * ct_w, fn * ct_w * 8,
                                             cudaMemcpyHostToDevice, cr->st));
                }
            };
            if (chunked) {
                for (int c = 0; c < n_chunks; c++) {
                    const int fb = c * kChunk, fn = std::min(kChunk, F - fb);
                    stage(fb, fn);
                    CUDA_TRY(cudaEventRecord(cr->ev[c], cr->st));
                }
            } else {
                stage(0, nb);
                CUDA_TRY(cudaEventRecord(cr->ev[0], cr->st));
                CUDA_TRY(cudaStreamWaitEvent(ctx->stream, cr->ev[0], 0));
                if (seed) kern::expand_uniform(ctx, ctx->stream, d, ct_w, c0s, nb, nl0, *seed, 0);
            }
            X = d;
        } else if (seed) {   // device c0: expanded into the staging buffer in stream order
            u64 *d = (u64 *)ctx->buf("layer_in", in_w * 8);
            kern::expand_uniform(ctx, ctx->stream, d, ct_w, in_cts, nb, nl0, *seed, 0);
            X = d;
        }
        // the staged inputs have been read (by the combination's kernels)
        auto inputs_read = [&]() {
            if (!cr) return;
            CUDA_TRY(cudaEventRecord(cr->free_ev, ctx->stream));
            cr->have_free = ctx->in_batch;
        };
        const int l1 = l0 - 1, LS = l1 + 1;           // lanes keep a fixed limb stride
        const size_t lane_w = (size_t)Fp * 2 * LS * N;
        const int max_lanes = std::max(1, pl->max_lanes);
        std::vector<u64 *> bufA(max_lanes), bufB(max_lanes);
        for (int i = 0; i < max_lanes; i++) {
            bufA[i] = (u64 *)ctx->buf("lane_a" + std::to_string(i), lane_w * 8);
            bufB[i] = (u64 *)ctx->buf("lane_b" + std::to_string(i), lane_w * 8);
        }
        u64 *acc = (u64 *)ctx->buf("acc", lane_w * 8);
        u64 *acc_new = (u64 *)ctx->buf("acc_new", lane_w * 8);

        // ---- Inter-CA (the client sent one copy of X per neighbour slot k):
        // Z_k = X_k W for every copy, then out = sum_k mask_k (x) Z_k, rescale
        if (pl->n_copies) {
            const std::vector<int> pid_l1 = iota(LS);
            u64 *Zc = (u64 *)ctx->buf("comb_z", (size_t)Fp * 2 * nl0 * N * 8);
            CUDA_TRY(cudaMemsetAsync(acc, 0, lane_w * 8, ctx->stream));
            for (int k = 0; k < pl->n_copies; k++) {
                kern::comb_const_mac(ctx, X + (size_t)k * F * 2 * nl0 * N, F, Fp, l0, pl->d_comb, Zc, nl0);
                kern::rescale_coef(ctx, Zc, nl0, bufA[0], LS, Fp * 2, l0);
                kern::LimbSet z{bufA[0], LS, LS, Fp * 2, pid_l1};
                kern::ntt_fwd(ctx, z, z);
                kern::stay_mac(ctx, bufA[0], LS, Fp, l1, {{acc, pl->masks[k].d}}, LS);
            }
            inputs_read();
            kern::rescale_ntt(ctx, acc, LS, Fp * 2, l1);
            const int level = l1 - 1, nlo = level + 1;
            FG_CHECK(level == pl->out_level, FG_ELEVEL, "plan output level mismatch");
            std::vector<int> pidx(LS, -1);
            for (int i = 0; i < nlo; i++) pidx[i] = i;
            kern::LimbSet as{acc, LS, LS, Fp * 2, pidx};
            kern::ntt_inv(ctx, as, as);
            const size_t out_w = (size_t)Fp * 2 * nlo * N;
            u64 *o = is_dev(out_cts) ? out_cts : (u64 *)ctx->buf("layer_out", out_w * 8);
            kern::copy_limbs(ctx, acc, LS, o, nlo, Fp * 2, nlo);
            if (o != out_cts)
                CUDA_TRY(cudaMemcpyAsync(out_cts, o, out_w * 8, cudaMemcpyDeviceToHost, ctx->stream));
            if (sync) CUDA_TRY(cudaStreamSynchronize(ctx->stream));
            if (out_level) *out_level = level;
            return;
        }

        // ---- 1. combination
        const std::vector<int> pid_l1 = iota(LS);
        if (t == 1) {
            u64 *Zc = (u64 *)ctx->buf("comb_z", (size_t)Fp * 2 * nl0 * N * 8);
            if (chunked) {
                for (int c = 0; c < n_chunks; c++) {
                    CUDA_TRY(cudaStreamWaitEvent(ctx->stream, cr->ev[c], 0));
                    const int fb = c * kChunk, fe = std::min(F, (c + 1) * kChunk);
                    if (seed)
                        kern::expand_uniform(ctx, ctx->stream, const_cast<u64 *>(X) + fb * ct_w, ct_w,
                                             c0s + fb * c0_w, fe - fb, nl0, *seed, (u64)fb);
                    kern::comb_const_mac(ctx, X, F, Fp, l0, pl->d_comb, Zc, nl0, fb, fe, c > 0);
                }
            } else {
                kern::comb_const_mac(ctx, X, F, Fp, l0, pl->d_comb, Zc, nl0);
            }
            inputs_read();
            kern::rescale_coef(ctx, Zc, nl0, bufA[0], LS, Fp * 2, l0);
            kern::LimbSet z{bufA[0], LS, LS, Fp * 2, pid_l1};
            kern::ntt_fwd(ctx, z, z);
        } else {
            const std::vector<int> pid0 = iota(nl0);
            u64 *Xn = (u64 *)ctx->buf("comb_xn", in_w * 8);
            kern::LimbSet xs{const_cast<u64 *>(X), nl0, nl0, nb * 2, pid0}, xd{Xn, nl0, nl0, nb * 2, pid0};
            kern::ntt_fwd(ctx, xs, xd);
            inputs_read();
            u64 *Za = (u64 *)ctx->buf("comb_acc", (size_t)Fp * 2 * nl0 * N * 8);
            CUDA_TRY(cudaMemsetAsync(Za, 0, (size_t)Fp * 2 * nl0 * N * 8, ctx->stream));
            for (int b = 0; b < nb; b++) {
                std::vector<kern::Dest> ds;
                for (int j = 0; j < Fp; j++)
                    ds.push_back({Za + (size_t)j * 2 * nl0 * N, pl->masks[pl->comb_masks[b][j]].d});
                kern::stay_mac(ctx, Xn + (size_t)b * 2 * nl0 * N, nl0, 1, l0, ds, nl0);
            }
            kern::rescale_ntt(ctx, Za, nl0, Fp * 2, l0);
            kern::copy_limbs(ctx, Za, nl0, bufA[0], LS, Fp * 2, LS);
            u64 *digits = (u64 *)ctx->buf("digits", (size_t)Fp * ctx->n_digits(l1) * ctx->ext(l1) * N * 8);
            u64 *tmp = acc_new;
            for (int k : pl->comb_rots) {
                kern::modup(ctx, bufA[0], LS, Fp, l1, digits);
                kern::rotate_mac(ctx, keys->get(((k % M) + M) % M), bufA[0], LS, Fp, l1, digits,
                                 {{tmp, nullptr}}, LS);
                kern::add(ctx, bufA[0], tmp, bufA[0], Fp * 2 * LS, pid_l1);
            }
        }

        // ---- 2. SpIntra-CA groups (one ModDown per output, see k_group_mac)
        std::vector<u64 *> *in = &bufA, *outb = &bufB;
        bool have_acc = false;
        int level = l1;
        const size_t ext_w = (size_t)Fp * 2 * ctx->ext(l1) * N;
        std::vector<u64 *> upool;
        for (const GroupC &g : pl->groups) {
            FG_CHECK(g.level == level, FG_ELEVEL, "plan level mismatch");
            // outputs: lanes 0..n_out-1, then the accumulator if the group feeds it
            bool any_acc = false;
            for (const TermC &tm : g.terms) any_acc |= tm.dst < 0;
            const int X = g.n_out + (any_acc ? 1 : 0);
            std::vector<u64 *> ext(X);
            for (int x = 0; x < X; x++) ext[x] = (u64 *)ctx->buf("ext" + std::to_string(x), ext_w * 8);
            auto out_index = [&](int dst) { return dst < 0 ? g.n_out : dst; };
            // terms by source: (lane, k) in plan order of the rotations, kept lanes after
            std::map<std::pair<int, int>, std::vector<const TermC *>> by_src;
            for (const TermC &tm : g.terms) by_src[{tm.src, tm.k}].push_back(&tm);
            // sources per launch: the group's sources split evenly over the
            // fewest launches within the program limits of k_group_mac (the
            // key-switch outputs of one launch are held at once)
            const int n_src = (int)by_src.size();
            const int n_launch = std::max({1, (n_src + kern::kGmacSrc - 1) / kern::kGmacSrc,
                                           ((int)g.terms.size() + kern::kGmacTerms - 1) / kern::kGmacTerms});
            const int per_launch = (n_src + n_launch - 1) / n_launch;
            u64 *digits = (u64 *)ctx->buf("digits",
                                          (size_t)Fp * ctx->n_digits(level) * ctx->ext(level) * N * 8);
            std::vector<kern::GroupSource> srcs;
            std::vector<kern::Dest> terms;
            std::vector<int> tdest;
            bool first_flush = true;
            std::vector<int> dest_terms(X, 0);   // terms per output since the last flush
            auto add_source = [&](const u64 *u, const u64 *lane, uint32_t galois,
                                  const std::vector<const TermC *> &ts) {
                for (const TermC *tm : ts) dest_terms[out_index(tm->dst)]++;
                kern::GroupSource gs{u, lane, galois, (int)terms.size(), 0};
                for (const TermC *tm : ts) {
                    terms.push_back({nullptr, pl->masks[tm->mask].d});
                    tdest.push_back(out_index(tm->dst));
                }
                gs.t1 = (int)terms.size();
                srcs.push_back(gs);
            };
            // key switches of the current lane not yet launched (one launch per
            // lane and pool, see ks_multi)
            std::vector<const KeyDev *> pend_keys;
            std::vector<u64 *> pend_u;
            const u64 *pend_lane = nullptr;
            auto issue_pending = [&]() {
                if (!pend_keys.empty())
                    kern::ks_multi(ctx, pend_keys, pend_u, pend_lane, LS, Fp, level, digits);
                pend_keys.clear();
                pend_u.clear();
            };
            auto flush = [&]() {
                issue_pending();
                if (srcs.empty()) return;
                // outputs in slices of at most 64 (the program's output table)
                for (int x0 = 0; x0 < X; x0 += 64) {
                    const int xn = std::min(64, X - x0);
                    std::vector<kern::GroupSource> ss;
                    std::vector<kern::Dest> tt;
                    std::vector<int> td;
                    for (const auto &gs : srcs) {
                        kern::GroupSource g2 = gs;
                        g2.t0 = (int)tt.size();
                        for (int t = gs.t0; t < gs.t1; t++)
                            if (tdest[t] >= x0 && tdest[t] < x0 + xn) {
                                tt.push_back(terms[t]);
                                td.push_back(tdest[t] - x0);
                            }
                        g2.t1 = (int)tt.size();
                        if (g2.t1 > g2.t0) ss.push_back(g2);
                    }
                    std::vector<u64 *> oo(ext.begin() + x0, ext.begin() + x0 + xn);
                    if (ss.empty() && first_flush) {
                        for (u64 *o : oo) CUDA_TRY(cudaMemsetAsync(o, 0, ext_w * 8, ctx->stream));
                        continue;
                    }
                    if (!ss.empty()) kern::group_mac(ctx, ss, tt, td, oo, !first_flush, Fp, level, LS);
                }
                first_flush = false;
                srcs.clear();
                terms.clear();
                tdest.clear();
                std::fill(dest_terms.begin(), dest_terms.end(), 0);
            };
            auto needs_flush = [&](const std::vector<const TermC *> &ts) {
                bool full = (int)srcs.size() >= per_launch ||
                            (int)(terms.size() + ts.size()) > kern::kGmacTerms;
                for (const TermC *tm : ts) full |= dest_terms[out_index(tm->dst)] >= 255;
                return full;
            };
            // kept values first (no key switching)
            for (auto &kv : by_src)
                if (kv.first.second == 0) {
                    if (needs_flush(kv.second)) flush();
                    add_source(nullptr, (*in)[kv.first.first], 0, kv.second);
                }
            int cur = -1, used = 0;
            for (auto &rk : g.rots) {
                const int a = rk.first, k = rk.second;
                auto it = by_src.find({a, k});
                if (it == by_src.end()) continue;
                if (needs_flush(it->second)) {
                    flush();
                    used = 0;
                }
                if (a != cur) {
                    issue_pending();   // the ModUp below overwrites the digits
                    kern::modup(ctx, (*in)[a], LS, Fp, level, digits);
                    cur = a;
                }
                if ((int)upool.size() <= used)
                    upool.push_back((u64 *)ctx->buf("upool" + std::to_string(used), ext_w * 8));
                const KeyDev &key = keys->get(((k % M) + M) % M);
                pend_keys.push_back(&key);
                pend_u.push_back(upool[used]);
                pend_lane = (*in)[a];
                add_source(upool[used], (*in)[a], key.galois, it->second);
                used++;
            }
            flush();
            // one ModDown per output, then the rescale that closes the group
            for (int x = 0; x < g.n_out; x++)
                kern::moddown_rescale_to_lane(ctx, ext[x], Fp, level, (*outb)[x], LS);
            if (any_acc) {
                kern::moddown_rescale_to_lane(ctx, ext[g.n_out], Fp, level, acc_new, LS);
                if (have_acc) {
                    std::vector<int> pidx(LS, -1);
                    for (int i = 0; i < level; i++) pidx[i] = i;
                    kern::add(ctx, acc, acc_new, acc, Fp * 2 * LS, pidx);
                } else {
                    std::swap(acc, acc_new);
                    have_acc = true;
                }
            }
            std::swap(in, outb);
            level--;
        }
        FG_CHECK(have_acc, FG_EINVAL, "the plan produced no output term");
        FG_CHECK(level == pl->out_level, FG_ELEVEL, "plan output level mismatch");

        // ---- 3. back to the coefficient domain, compact [Fp][2][level+1][N]
        const int nlo = level + 1;
        std::vector<int> pidx(LS, -1);
        for (int i = 0; i < nlo; i++) pidx[i] = i;
        kern::LimbSet as{acc, LS, LS, Fp * 2, pidx};
        kern::ntt_inv(ctx, as, as);
        const size_t out_w = (size_t)Fp * 2 * nlo * N;
        u64 *o = is_dev(out_cts) ? out_cts : (u64 *)ctx->buf("layer_out", out_w * 8);
        kern::copy_limbs(ctx, acc, LS, o, nlo, Fp * 2, nlo);
        if (o != out_cts)
            CUDA_TRY(cudaMemcpyAsync(out_cts, o, out_w * 8, cudaMemcpyDeviceToHost, ctx->stream));
        if (sync) CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        if (out_level) *out_level = level;
    }
}

// ------------------------------------------------------------------ batched layers
// Several layers (queries with their own plans) in flight at once: query q
// runs on stream q mod S with its own workspace, between a fork and a join
// on the context's stream.  Every query runs exactly the kernels it would
// run alone, so the results do not depend on S or on the graph.
static void batch_pass(fg_ctx *ctx, const fg_keys *keys, const fg_plan *const *plans, int n,
                       const uint64_t *const *in_cts, uint64_t *const *out_cts, int S,
                       int *levels)
{
    while ((int)ctx->pool.size() < S) {
        cudaStream_t st;
        CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        ctx->pool.push_back(st);
    }
    while ((int)ctx->pool_events.size() < S + 1) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->pool_events.push_back(e);
    }
    cudaStream_t origin = ctx->stream;
    CUDA_TRY(cudaEventRecord(ctx->pool_events[S], origin));
    for (int s = 0; s < S; s++) CUDA_TRY(cudaStreamWaitEvent(ctx->pool[s], ctx->pool_events[S], 0));
    for (auto &kv : ctx->copies) kv.second.have_free = false;
    ctx->in_batch = true;
    try {
        for (int q = 0; q < n; q++) {
            const fg_plan *pl = plans[q];
            ctx->stream = ctx->pool[q % S];
            ctx->ws_prefix = "b" + std::to_string(q % S) + "/";
            const int nb = pl->n_copies ? pl->n_copies * pl->F : pl->t == 1 ? pl->F : (pl->F + pl->t - 1) / pl->t;
            layer_exec(ctx, keys, pl, in_cts[q], nb, out_cts[q], pl->Fp, false, &levels[q],
                       ctx->batch_seeds ? &ctx->batch_seeds[q] : nullptr);
        }
    } catch (...) {
        ctx->stream = origin;
        ctx->ws_prefix.clear();
        ctx->in_batch = false;
        throw;
    }
    ctx->stream = origin;
    ctx->ws_prefix.clear();
    ctx->in_batch = false;
    for (auto &kv : ctx->copies) kv.second.have_free = false;
    for (int s = 0; s < S; s++) {
        CUDA_TRY(cudaEventRecord(ctx->pool_events[s], ctx->pool[s]));
        CUDA_TRY(cudaStreamWaitEvent(origin, ctx->pool_events[s], 0));
    }
}

static double time_pass(fg_ctx *ctx, const fg_keys *keys, const fg_plan *const *plans, int n,
                        const uint64_t *const *in_cts, uint64_t *const *out_cts, int S, int *levels)
{
    cudaEvent_t a, b;
    CUDA_TRY(cudaEventCreate(&a));
    CUDA_TRY(cudaEventCreate(&b));
    CUDA_TRY(cudaEventRecord(a, ctx->stream));
    batch_pass(ctx, keys, plans, n, in_cts, out_cts, S, levels);
    CUDA_TRY(cudaEventRecord(b, ctx->stream));
    CUDA_TRY(cudaEventSynchronize(b));
    float ms = 0;
    CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

// the batch runs from ctx->batch_stream (a non-blocking stream that can be
// captured, which the legacy default stream cannot), joined to ctx->stream
// before and after
// the kernels' launch configuration for the batch, chosen by timing whole
// passes on one stream: coordinate descent over the knobs of Tune, each
// candidate timed twice (the faster counts), from the defaults
static void tune_batch(fg_ctx *ctx, const fg_keys *keys, const fg_plan *const *plans, int n,
                       const uint64_t *const *in_cts, uint64_t *const *out_cts, int *levels)
{
    ctx->tune_ms.clear();
    Tune best = ctx->tune;
    auto timed = [&](const Tune &t) {
        ctx->tune = t;
        double ms = 0;
        for (int rep = 0; rep < 2; rep++) {
            const double m = time_pass(ctx, keys, plans, n, in_cts, out_cts, 1, levels);
            ms = rep == 0 ? m : std::min(ms, m);
        }
        ctx->tune_ms.push_back(ms);
        return ms;
    };
    double best_ms = timed(best);
    const int cols[2] = {16, 8}, rows[2] = {16, 8}, tw[2] = {0, 1}, split[3] = {0, 1, 2}, kcols[2] = {1, 2},
              fused[2] = {0, 1}, groups[3] = {7, 4, 13};
    const int dfused[2] = {0, 1}, gregs[2] = {0, 1}, kara[2] = {0, 1};
    auto knob = [&](auto field, const int *vals, int nv) {
        Tune base = best;
        for (int k = 0; k < nv; k++) {
            Tune t = base;
            t.*field = vals[k];
            if (t == base) continue;
            const double ms = timed(t);
            if (ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
    };
    if (ctx->log_n == 16) {
        knob(&Tune::ntt_cols, cols, 2);
        knob(&Tune::ntt_rows, rows, 2);
        knob(&Tune::ntt_tw, tw, 2);
        knob(&Tune::modup_fused, fused, 2);
        knob(&Tune::moddown_fused, dfused, 2);
    }
    knob(&Tune::ks_split, split, 3);
    knob(&Tune::ks_cols, kcols, 2);
    knob(&Tune::gmac_groups, groups, 3);
    knob(&Tune::kara, kara, 2);
    knob(&Tune::gmac_regs, gregs, 2);
    ctx->batch_tune = best;
    ctx->batch_tuned = true;
}

static void batch_body(fg_ctx *ctx, const fg_keys *keys, const fg_plan *const *plans, int n,
                       const uint64_t *const *in_cts, uint64_t *const *out_cts, const fg_batch_opts &o,
                       const std::vector<const void *> &args, int *out_levels, int *streams_used)
{
    // replay the captured batch when the arguments are the same
    if (o.graph && ctx->batch.exec && ctx->batch.args == args &&
        (o.streams == 0 || o.streams == ctx->batch.streams)) {
        CUDA_TRY(cudaGraphLaunch(ctx->batch.exec, ctx->stream));
        ctx->launches += ctx->batch.launches;
        for (int q = 0; q < n; q++) out_levels[q] = plans[q]->out_level;
        if (streams_used) *streams_used = ctx->batch.streams;
        return;
    }
    // the batch's launch configuration stays in force for this call only
    struct KeepTune {
        fg_ctx *c;
        Tune t;
        ~KeepTune() { c->tune = t; }
    } keep{ctx, ctx->tune};
    if (o.tune && !ctx->batch_tuned) {
        batch_pass(ctx, keys, plans, n, in_cts, out_cts, 1, out_levels);   // workspaces, warm-up
        CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        tune_batch(ctx, keys, plans, n, in_cts, out_cts, out_levels);
    }
    if (o.tune && ctx->batch_tuned) ctx->tune = ctx->batch_tune;
    // first call: one pass with every workspace allocated (this pass gives
    // the results), then the stream count, then the capture
    int S = o.streams ? std::min(o.streams, n) : 1;
    if (o.streams == 0) {
        // every stream needs a workspace like stream 0's: as many streams as
        // the free device memory holds (with a margin), at most 8
        batch_pass(ctx, keys, plans, n, in_cts, out_cts, 1, out_levels);
        CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        size_t per_stream = 0, free_b = 0, total_b = 0;
        for (const auto &kv : ctx->ws)
            if (kv.first.rfind("b0/", 0) == 0) per_stream += kv.second.second;
        CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
        const int smax = (int)std::max<size_t>(
            1, std::min<size_t>(8, 1 + (size_t)(0.8 * (double)free_b) / std::max<size_t>(per_stream, 1)));
        // the largest candidate first, so that every workspace exists
        // before the timed passes
        const int cand[4] = {8, 4, 2, 1};
        int top = 1;
        for (int c : cand)
            if (c <= n && c <= smax) {
                top = c;
                break;
            }
        batch_pass(ctx, keys, plans, n, in_cts, out_cts, top, out_levels);
        CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        double best = 0;
        for (int c : cand) {
            if (c > top) continue;
            const double ms = time_pass(ctx, keys, plans, n, in_cts, out_cts, c, out_levels);
            if (best == 0 || ms < best) {
                best = ms;
                S = c;
            }
        }
    } else {
        batch_pass(ctx, keys, plans, n, in_cts, out_cts, S, out_levels);
    }
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (o.graph) {
        if (ctx->batch.exec) {
            cudaGraphExecDestroy(ctx->batch.exec);
            ctx->batch.exec = nullptr;
        }
        const int64_t l0 = ctx->launches;
        cudaGraph_t g = nullptr;
        CUDA_TRY(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed));
        try {
            batch_pass(ctx, keys, plans, n, in_cts, out_cts, S, out_levels);
        } catch (...) {
            cudaStreamEndCapture(ctx->stream, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        CUDA_TRY(cudaStreamEndCapture(ctx->stream, &g));
        cudaGraphExec_t ex = nullptr;
        const cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) throw fg_error(FG_ECUDA, std::string("graph: ") + cudaGetErrorString(e));
        ctx->batch.exec = ex;
        ctx->batch.args = args;
        ctx->batch.streams = S;
        ctx->batch.launches = ctx->launches - l0;
        ctx->launches = l0;
    }
    if (streams_used) *streams_used = S;
}

extern "C" int fg_batch_tuning(const fg_ctx *ctx, int cfg[10], double *ms, int cap, int *n)
{
    if (!ctx || !cfg || !n || cap < 0) return FG_EINVAL;
    const Tune &t = ctx->batch_tuned ? ctx->batch_tune : ctx->tune;
    cfg[0] = t.ntt_cols;
    cfg[1] = t.ntt_rows;
    cfg[2] = t.ntt_tw;
    cfg[3] = t.ks_split;
    cfg[4] = t.ks_cols;
    cfg[5] = t.modup_fused;
    cfg[6] = t.moddown_fused;
    cfg[7] = t.gmac_groups;
    cfg[8] = t.gmac_regs;
    cfg[9] = t.kara;
    *n = ctx->batch_tuned ? (int)ctx->tune_ms.size() : 0;
    if (ms)
        for (int i = 0; i < std::min(cap, *n); i++) ms[i] = ctx->tune_ms[i];
    return FG_OK;
}

extern "C" int fg_ctx_set_tuning(fg_ctx *ctx, const int cfg[10])
{
    if (!ctx || !cfg) return FG_EINVAL;
    if ((cfg[0] != 16 && cfg[0] != 8) || (cfg[1] != 16 && cfg[1] != 8) || (cfg[2] != 0 && cfg[2] != 1) ||
        (cfg[3] < 0 || cfg[3] > 2) || (cfg[4] != 1 && cfg[4] != 2) || (cfg[5] != 0 && cfg[5] != 1) ||
        (cfg[6] != 0 && cfg[6] != 1) || cfg[7] < 1 || (cfg[8] != 0 && cfg[8] != 1) ||
        (cfg[9] != 0 && cfg[9] != 1))
        return FG_EINVAL;
    ctx->tune.ntt_cols = cfg[0];
    ctx->tune.ntt_rows = cfg[1];
    ctx->tune.ntt_tw = cfg[2];
    ctx->tune.ks_split = cfg[3];
    ctx->tune.ks_cols = cfg[4];
    ctx->tune.modup_fused = cfg[5];
    ctx->tune.moddown_fused = cfg[6];
    ctx->tune.gmac_groups = cfg[7];
    ctx->tune.gmac_regs = cfg[8];
    ctx->tune.kara = cfg[9];
    return FG_OK;
}

static int layer_batch(fg_ctx *ctx, const fg_keys *keys, const fg_plan *const *plans, int n,
                       const uint64_t *const *in_cts, const uint64_t *seeds, uint64_t *const *out_cts,
                       const fg_batch_opts *opts, int *out_levels, int *streams_used)
{
    if (!ctx) return FG_EINVAL;
    cudaStream_t home = ctx->stream;
    struct KeepSeeds {
        fg_ctx *c;
        ~KeepSeeds() { c->batch_seeds = nullptr; }
    } keep{ctx};
    ctx->batch_seeds = seeds;
    try {
        FG_CHECK(keys && plans && in_cts && out_cts && out_levels && n >= 1, FG_EINVAL, "null argument");
        fg_batch_opts o{0, 1, 0};
        if (opts) o = *opts;
        FG_CHECK(o.streams >= 0 && o.streams <= 16, FG_EINVAL, "streams must be 0..16");
        std::vector<const void *> args;
        for (int q = 0; q < n; q++) {
            FG_CHECK(plans[q] && plans[q]->ctx == ctx && keys->ctx == ctx, FG_EINVAL,
                     "plan or keys of another context");
            FG_CHECK(in_cts[q] && out_cts[q] && (is_dev(in_cts[q]) || is_pinned(in_cts[q])) && is_dev(out_cts[q]),
                     FG_EINVAL, "batched layers take device or page-locked host inputs and device outputs");
            args.insert(args.end(), {plans[q], in_cts[q], out_cts[q]});
            if (seeds) args.push_back(reinterpret_cast<const void *>(static_cast<uintptr_t>(seeds[q])));
        }
        args.push_back(seeds ? &ctx->batch_seeds : nullptr);   // seeded and full batches never match
        if (!ctx->batch_stream)
            CUDA_TRY(cudaStreamCreateWithFlags(&ctx->batch_stream, cudaStreamNonBlocking));
        CUDA_TRY(cudaStreamSynchronize(home));   // inputs written on the caller's stream
        ctx->stream = ctx->batch_stream;
        batch_body(ctx, keys, plans, n, in_cts, out_cts, o, args, out_levels, streams_used);
        CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        ctx->stream = home;
    } catch (const fg_error &e) {
        ctx->stream = home;
        ctx->err = e.what();
        return e.code;
    } catch (const std::exception &e) {
        ctx->stream = home;
        ctx->err = e.what();
        return FG_EOOM;
    }
    return FG_OK;
}

extern "C" int fg_gcn_layer_batch(fg_ctx *ctx, const fg_keys *keys, const fg_plan *const *plans, int n,
                                  const uint64_t *const *in_cts, uint64_t *const *out_cts,
                                  const fg_batch_opts *opts, int *out_levels, int *streams_used)
{
    return layer_batch(ctx, keys, plans, n, in_cts, nullptr, out_cts, opts, out_levels, streams_used);
}

extern "C" int fg_gcn_layer_batch_seeded(fg_ctx *ctx, const fg_keys *keys, const fg_plan *const *plans, int n,
                                         const uint64_t *const *in_c0, const uint64_t *seeds,
                                         uint64_t *const *out_cts, const fg_batch_opts *opts, int *out_levels,
                                         int *streams_used)
{
    if (!ctx) return FG_EINVAL;
    if (!seeds) {
        ctx->err = "null seeds";
        return FG_EINVAL;
    }
    return layer_batch(ctx, keys, plans, n, in_c0, seeds, out_cts, opts, out_levels, streams_used);
}

extern "C" {

int fg_gcn_layer_axw_seeded(fg_ctx *ctx, const fg_keys *keys, const fg_plan *pl, const uint64_t *in_c0,
                            int n_in, uint64_t seed, uint64_t *out_cts, int n_out, int *out_level,
                            double *out_scale)
{
    if (!ctx) return FG_EINVAL;
    try {
        layer_exec(ctx, keys, pl, in_c0, n_in, out_cts, n_out, true, out_level, &seed);
        if (out_scale) *out_scale = ctx->scale;
    } catch (const fg_error &e) {
        ctx->err = e.what();
        return e.code;
    } catch (const std::exception &e) {
        ctx->err = e.what();
        return FG_EOOM;
    }
    return FG_OK;
}

int fg_gcn_layer_axw(fg_ctx *ctx, const fg_keys *keys, const fg_plan *pl, const uint64_t *in_cts,
                     int n_in, uint64_t *out_cts, int n_out, int *out_level, double *out_scale)
{
    if (!ctx) return FG_EINVAL;
    try {
        layer_exec(ctx, keys, pl, in_cts, n_in, out_cts, n_out, true, out_level);
        if (out_scale) *out_scale = ctx->scale;
    } catch (const fg_error &e) {
        ctx->err = e.what();
        return e.code;
    } catch (const std::exception &e) {
        ctx->err = e.what();
        return FG_EOOM;
    }
    return FG_OK;
}

}  // extern "C"
