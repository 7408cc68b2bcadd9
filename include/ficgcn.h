/*
 * ficgcn.h -- C ABI of a GB300 (sm_103a) library for one encrypted GCN layer
 * A-hat * X * W under CKKS, following FicGCN (Kan et al., ICML 2025).
 *
 * Problem statement (paper Sec. 1 and Sec. 2.4, threat model): the server
 * holds the plaintext normalised adjacency A-hat and weights W; the client
 * holds the secret key and sends Enc(X); the server returns Enc(A-hat X W),
 * which only the client can decrypt.  The server computes the combination
 * X W first (latency-aware column packing, Sec. 3.2 / App. B.1) and then the
 * sparse aggregation by SpIntra-CA rotate-and-sum (Sec. 3.3) over a node
 * order chosen on the server and propagated back to the client packer
 * (App. B.2).
 *
 * Conventions shared by every call
 *   - Status: every call returns an int, FG_OK (0) or a negative FG_E* code.
 *     fg_last_error(ctx) gives the text of the last failure on that context.
 *     No C++ exception crosses this boundary.
 *   - Ring: N = 2^log_n, M = N/2 slots; primes q_0..q_L (ciphertext modulus)
 *     and p_0..p_{K-1} (special primes of key switching); level l means the
 *     ciphertext lives modulo q_0..q_l.
 *   - Ciphertexts cross the boundary as uint64 [2][l+1][N], limb-major,
 *     COEFFICIENT domain, every residue canonical in [0, q_i).  A batch of
 *     ciphertexts is contiguous.  Plaintexts are uint64 [l+1][N], same rules.
 *   - Buffers: every uint64_t* ciphertext/plaintext argument may point to
 *     host or device memory (the library asks the CUDA runtime which).  The
 *     caller owns every buffer it passes; the library owns handles (fg_ctx,
 *     fg_keys, fg_plan) and the device copies of keys and plans.  Blobs
 *     returned by the library are freed with fg_free.
 *   - Streams: the CUDA stream given at context creation carries every
 *     kernel and copy of that context; calls return once their results are
 *     in the caller's buffers (device outputs: complete on that stream).
 *   - Randomness (keys, encryption): SplitMix64 (Steele, Lea & Flood,
 *     OOPSLA 2014).  Stream (seed, purpose, index) starts from the state
 *     mix(seed ^ (purpose << 48) ^ index), mix being SplitMix64's output
 *     function; each draw adds 0x9E3779B97F4A7C15 to the state and returns
 *     mix(state).  Ternary coefficient: draw >> 62, redrawn while 3, minus 1.
 *     Noise coefficient: the discrete Gaussian sigma = 3.2 cut at |x| <= 19,
 *     by inversion of the table T[k] = floor(2^63 sum_{i<=k} p_i / S) over
 *     |x| (p_0 = rho(0), p_i = 2 rho(i), rho(x) = exp(-x^2 / (2 sigma^2)),
 *     S = sum p_i): |x| = least k with (d >> 1) < T[k], sign from bit 0 of
 *     d (zero has no sign).  Uniform residue mod q:
 *     d & (2^bitlen(q) - 1), redrawn while >= q; limbs in prime order.
 *     Purposes: 1 secret (index 0), 2/3 key a/e (index galois << 8 | digit),
 *     4/5 encryption a/e (index = ciphertext index).  This generator is not
 *     cryptographic; it makes every run reproducible.
 */
#ifndef FICGCN_H
#define FICGCN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FG_OK 0
#define FG_EINVAL (-1)    /* bad argument, shape or size */
#define FG_ELEVEL (-2)    /* level/scale mismatch, level budget exhausted */
#define FG_EKEY (-3)      /* missing rotation key, bad blob or checksum */
#define FG_ECUDA (-4)     /* a CUDA runtime call failed */
#define FG_EOOM (-5)      /* device or host allocation failed */
#define FG_ETIMEOUT (-6)  /* a bounded device wait ran out */
#define FG_ENODEV (-7)    /* no usable CUDA device */

typedef struct fg_ctx fg_ctx;
typedef struct fg_keys fg_keys;
typedef struct fg_plan fg_plan;

/* RNS-CKKS parameters (paper Sec. 2.1: Q = prod q_i, L levels).
 * Primes: for each bit size, in the order q_bits then p_bits, the largest
 * prime below 2^bits that is 1 mod 2N and not taken before.  alpha primes
 * form one key-switching digit (hybrid key switching).  10 <= log_n <= 16,
 * 2 <= n_q <= 60, 1 <= n_p <= 7, bit sizes in [log_n + 2, 60], at most 16
 * digits (ceil(n_q / alpha)). */
typedef struct {
    int log_n;
    int n_q;
    const int *q_bits;
    int n_p;
    const int *p_bits;
    int alpha;
    double log_scale;   /* Delta = 2^log_scale */
} fg_params;

/* ---------------------------------------------------------------- context */

/* Create a context on the current CUDA device.  cuda_stream: a cudaStream_t
 * (NULL = the legacy default stream).  Builds the primes, NTT tables and
 * RNS constants on the device.  FG_ENODEV without a device. */
int fg_ctx_create(const fg_params *params, void *cuda_stream, fg_ctx **out);
int fg_ctx_destroy(fg_ctx *ctx);
/* ctx == NULL: the text of the last failed fg_ctx_create. */
const char *fg_last_error(const fg_ctx *ctx);
/* q_out: n_q primes, p_out: n_p primes (host arrays). */
int fg_ctx_primes(const fg_ctx *ctx, uint64_t *q_out, uint64_t *p_out);
/* Device memory the context holds now (tables + workspace), in bytes. */
int fg_ctx_device_bytes(const fg_ctx *ctx, size_t *bytes);
void fg_free(void *blob);

/* Instrumentation (no counterpart in the paper, which times on one CPU
 * thread).  fg_ctx_time_kernels: from now on record a CUDA event pair on the
 * context's stream around every call of one kernel class -- "ntt" (one call
 * = the two kernels of a batched transform), "ks_ip", "moddown_conv",
 * "moddown_mac", "modup_conv", "comb", "rescale", "stay_mac" -- with the
 * call's algorithmic bytes (each operand read once, each result written
 * once); NULL or "" stops.  Earlier records are dropped.
 * fg_ctx_kernel_times: waits for the stream, returns the summed device time
 * in ms, the number of calls and their algorithmic bytes, and clears the
 * records.  fg_ctx_launch_count: kernels this context has launched so far. */
int fg_ctx_time_kernels(fg_ctx *ctx, const char *kernel_class);
int fg_ctx_kernel_times(fg_ctx *ctx, double *ms, int64_t *calls, double *alg_bytes);
int fg_ctx_launch_count(const fg_ctx *ctx, int64_t *launches);
/* Wait for the device, then free the context's workspace (the scratch
 * buffers its calls grow on demand and keep for reuse); later calls
 * allocate again.  Keys, plans and tables stay. */
int fg_ctx_release_workspace(fg_ctx *ctx);

/* ---------------------------------------------------------------- client */

/* Secret key and rotation keys (paper Sec. 2.1: Rot needs a key per amount).
 * Rotation amount k (left rotation by k slots, Rot(v, k) = (v_k, ..,
 * v_{M-1}, v_0, .., v_{k-1})) uses the Galois element g = 5^(k mod M) mod
 * 2N.  Each key switches phi_g(s) -> s with hybrid digits: for top-level
 * digit D_j, b_j = -a_j s + e_j + P [q_i in D_j] phi_g(s) mod q_i and
 * b_j = -a_j s + e_j mod p_k.  Blobs (host memory, free with fg_free) are
 * versioned, checksummed and hold keys in the coefficient domain. */
int fg_keygen(fg_ctx *ctx, uint64_t seed, const int32_t *rot_amounts, int n_rot, int relin,
              void **sk_blob, size_t *sk_len, void **evk_blob, size_t *evk_len);
/* With relin = 1 fg_keygen also makes the relinearisation key (for the
 * ciphertext product CMult of Sec. 2.1): the same construction switching
 * s^2 -> s, sampled with stream index 0 (Galois elements, the indices of the
 * rotation keys, are odd).  It is stored in the evk blob as amount FG_RELIN
 * with Galois element 1. */
#define FG_RELIN (-1)

/* CKKS encoding (canonical embedding, paper Sec. 2.1): real slot values
 * z_0..z_{n_slots-1} (missing slots are 0) -> coefficients m with
 * m(zeta^(5^j)) ~ scale * z_j, zeta = exp(i pi/N), rounded half away from
 * zero, reduced mod q_0..q_level into out [level+1][N].  FP64 on the host. */
int fg_encode_plain(fg_ctx *ctx, const double *slots, int n_slots, double scale,
                    int level, uint64_t *out);

/* Secret-key encryption of a plaintext at a level: c = (-a s + m + e, a),
 * a and e from streams (seed, 4/5, index).  pt: [level+1][N], out: [2][level+1][N]. */
int fg_encrypt(fg_ctx *ctx, const void *sk_blob, size_t sk_len, uint64_t seed,
               uint64_t index, const uint64_t *pt, int level, uint64_t *out);

/* Client packing (paper Sec. 3.2 and App. B.1, column-major packing of t
 * columns per ciphertext; App. B.2, node order from the server): X is
 * double [V][F] row-major; perm[v] in [0, M/t) is node v's slot; ciphertext
 * b holds column b*t + k in block k: slot k*(M/t) + perm[v].  Encoded at
 * Delta, encrypted at the top level with stream index b.  out_cts: room for
 * ceil(F/t) ciphertexts [2][L+1][N]; *n_out receives ceil(F/t). */
int fg_pack_features(fg_ctx *ctx, const void *sk_blob, size_t sk_len, uint64_t seed,
                     const double *X, int V, int F, const int32_t *perm, int t,
                     uint64_t *out_cts, int *n_out);

/* Seeded (compressed) client packing: the same packing and encryption, but
 * the uniform part a of ciphertext b is drawn from the stream (seed, 6, b)
 * coefficient by coefficient, (w_hi 2^64 + w_lo) mod q_i from the stream's
 * words 2(i N + x) and 2(i N + x) + 1, so that the receiver regenerates it
 * from (seed, b) alone; only c0 = -a s + m + e is written.  This is a
 * transport form of the paper's client-encrypted features (Sec. 3.2), half
 * the bytes of fg_pack_features.  out_c0 (host or device): room for
 * ceil(F/t) polynomials [L+1][N]; *n_out receives ceil(F/t). */
int fg_pack_features_seeded(fg_ctx *ctx, const void *sk_blob, size_t sk_len, uint64_t seed,
                            const double *X, int V, int F, const int32_t *perm, int t,
                            uint64_t *out_c0, int *n_out);

/* Full ciphertexts [n][2][level+1][N] of seeded ones 0..n-1 of a seed (c0:
 * [n][level+1][N]; host or device, either side): c1 of ciphertext b
 * regenerated on the device as fg_pack_features_seeded drew it.  FG_EINVAL
 * for n outside 0..65535 or level outside 0..L. */
int fg_expand_seeded(fg_ctx *ctx, uint64_t seed, const uint64_t *c0, int n, int level,
                     uint64_t *out_cts);

/* The client's Inter-CA input (paper Sec. 3.1: the node arrangements the
 * client encrypts offline): for every neighbour slot k < n, the rows
 * nbr[v][k] of X (zero where nbr is -1) packed as fg_pack_features does with
 * t = 1, copy k encrypted under seed + k.  nbr: [V][n] row-major; out_cts:
 * room for n*F ciphertexts [2][L+1][N], copy-major (copy k, column f at
 * k*F + f); host or device. */
int fg_pack_neighbor_copies(fg_ctx *ctx, const void *sk_blob, size_t sk_len, uint64_t seed,
                            const double *X, int V, int F, const int32_t *nbr, int n,
                            const int32_t *perm, uint64_t *out_cts);

/* Decryption m = c0 + c1 s mod q_i (paper Sec. 2.1).  out_pt: [level+1][N]. */
int fg_decrypt(fg_ctx *ctx, const void *sk_blob, size_t sk_len, const uint64_t *ct,
               int level, uint64_t *out_pt);

/* Decryption followed by decoding: out_slots receives the M real slot
 * values (imaginary parts dropped).  Needs |m| < q_0 q_1 / 2 (q_0 / 2 at
 * level 0) coefficient-wise, which holds for every ciphertext this library
 * produces at its scale. */
int fg_decrypt_decode(fg_ctx *ctx, const void *sk_blob, size_t sk_len, const uint64_t *ct,
                      int level, double scale, double *out_slots);

/* ---------------------------------------------------------------- server */

/* Copy the rotation keys of an evk blob to the device (NTT domain) after
 * checking its magic, parameters and checksum (FG_EKEY otherwise). */
int fg_load_evk(fg_ctx *ctx, const void *evk_blob, size_t len, fg_keys **out);
int fg_keys_destroy(fg_keys *keys);
/* Coefficient-domain copy of key `amount`'s digit j (amount FG_RELIN: the
 * relinearisation key): b and a as [L+1+K][N] (host or device buffers).
 * FG_EKEY if the amount has no key. */
int fg_keys_export(const fg_keys *keys, int32_t amount, int digit, uint64_t *b_out,
                   uint64_t *a_out);

typedef struct {
    int t;              /* columns per ciphertext; 0 = latency-aware rule J(t) */
    int radix_bits;     /* SpIntra-CA bits per group; 0 = fewest groups the budget allows */
    int aoo;            /* 1 = shortest cyclic shift (AOO), 0 = shift in [0, M) */
    int min_out_level;  /* lowest level the output may reach */
    int n_sampled;      /* n in J(t;F,n); 0 = mean row length of A-hat, rounded */
    int in_level;       /* level of the input ciphertexts; 0 = the top level L */
    int no_encode;      /* 1 = leave every mask zero (no encoding or upload): a plan
                           for timing only, whose layer computes nothing meaningful
                           (the kernels' work does not depend on the values) */
} fg_plan_opts;

/* Plan of one layer (paper Sec. 3.2-3.3): packing t, combination constants,
 * SpIntra-CA groups (per group: the rotations, the masked products into
 * lanes and into the accumulator), and every mask encoded at scale q_l on
 * the device.  A-hat: CSR (row_ptr [V+1], col, val), node v aggregating
 * column col[e] with weight val[e]; no repeated (row, col) pairs.  W: double
 * [F][Fp] row-major.  perm: node -> slot in [0, M/t) (injective).
 * Input ciphertexts are expected at the top level L.  opts may be NULL. */
int fg_plan_build(fg_ctx *ctx, const int32_t *row_ptr, const int32_t *col,
                  const double *val, int V, const double *W, int F, int Fp,
                  const int32_t *perm, const fg_plan_opts *opts, fg_plan **out);
int fg_plan_destroy(fg_plan *plan);

typedef struct {
    int t, B, n_in, n_out, in_level, out_level, n_groups, n_masks, n_keys;
    int64_t rotations;        /* complete Rot ops per layer call (all columns) */
    int64_t masked_products;  /* plaintext-ciphertext products per layer call */
} fg_plan_info_t;
int fg_plan_info(const fg_plan *plan, fg_plan_info_t *info);
/* The distinct rotation amounts (mod M) the plan needs keys for. */
int fg_plan_rotation_amounts(const fg_plan *plan, int32_t *out, int cap, int *n);
/* The plan's structure as int64 records: [N, M, t, B, V, F, Fp, in_level,
 * out_level, radix_bits, aoo, n_groups, n_masks], perm[V], the combination
 * (t == 1: F*Fp integer constants; t > 1: nb*Fp mask ids, n_rots, rots),
 * per group [bit_lo, n_bits, level, n_in, n_out, n_rots, (src, k)*,
 * n_terms, (src, k, dst, mask)*] (dst -1 = the accumulator), per mask
 * [level, n_slots, (slot, IEEE-754 bits of the value)*].
 * With out == NULL only *len is set. */
int fg_plan_describe(const fg_plan *plan, int64_t *out, size_t cap, size_t *len);
/* Host-only planning (no device, no context): the records fg_plan_describe
 * would give for the same inputs and parameters.  Lets a server plan
 * offline, e.g. to tell the client which rotation keys to generate before
 * any GPU work.  With out == NULL only *len is set. */
int fg_plan_dry_run(const fg_params *params, const int32_t *row_ptr, const int32_t *col,
                    const double *val, int V, const double *W, int F, int Fp,
                    const int32_t *perm, const fg_plan_opts *opts, int64_t *out, size_t cap,
                    size_t *len);
/* Node order optimisation (paper Sec. 3.4, Alg. 1), host only: perm_out[v]
 * receives the slot in [0, M) of node v of the graph A-hat (CSR row_ptr[V+1],
 * col; values not needed).  Regions of at most TH nodes found by a
 * breadth-first search over siblings (nodes with a common aggregation
 * target) from the highest-degree unplaced node; regions interleaved one
 * slot per turn, blanks taking the turns of exhausted regions while any of
 * the M - V remain; inside a region, nodes placed greedily at the free slot
 * with the fewest rotation steps (set bits of the index distances) to their
 * placed neighbours, ties to the lowest index.  *n_regions (may be NULL)
 * receives the number of regions.  FG_EINVAL for V < 1, M < V, TH < 1, or a
 * malformed CSR. */
int fg_node_order(const int32_t *row_ptr, const int32_t *col, int V, int M, int TH,
                  int32_t *perm_out, int *n_regions);
/* fg_node_order with a choice of the order in which the regions take their
 * turns in the interleaving (the paper leaves it open): region_order 0 =
 * the order the search found them (fg_node_order), 1 = larger regions first
 * (ties: search order). */
int fg_node_order_ex(const int32_t *row_ptr, const int32_t *col, int V, int M, int TH,
                     int region_order, int32_t *perm_out, int *n_regions);
/* Inter-CA plan (paper Sec. 3.1, Table 1; the first-layer mode): the client
 * sends n copies of X, copy k holding row nbr[v][k] of X at node v's slot
 * (fg_pack_features of the gathered rows; nbr -1: no neighbour), and the
 * server computes out_j = sum_k wts[.][k] (x) (X_k W)_j by PMult and Add
 * only (no rotation): the combination of every copy (constants at q_l),
 * a rescale, the masked sum over k (masks at q_{l-1}), a rescale.  nbr and
 * wts are [V][n] row-major; t = 1; the layer takes n*F input ciphertexts
 * (copy-major) and returns Fp at level in_level - 2.  GraphSage's MEAN over
 * {v} and n sampled neighbours is nbr[v] = (v, u_1, .., u_n), wts = 1/(n+1). */
int fg_plan_build_inter(fg_ctx *ctx, const int32_t *nbr, const double *wts, int V, int n,
                        const double *W, int F, int Fp, const int32_t *perm,
                        const fg_plan_opts *opts, fg_plan **out);

/* Aggregation mode of one layer (paper Sec. 3.4 "Selecting Aggregation
 * Mode", App. B.2, Table 1), host only like fg_plan_dry_run.  The
 * SpIntra-CA plan of (params, A-hat, W, perm, opts) is built and its
 * rotations R and masked terms T per output column counted; with n node
 * arrangements (n_copies: the largest row length of A-hat for the exact
 * layer, 1 + the sample size for GraphSage), F input columns and t columns
 * per ciphertext, the costs per output column are
 *   cost[0] SpIntra-CA = (ceil(F/t) + T)(L_pmult + L_add) + (ceil(log2 t) + R) L_rot,
 *   cost[1] Inter-CA   = (n ceil(F/t) + n)(L_pmult + L_add) + ceil(log2 t) L_rot,
 * lat = {L_rot, L_pmult, L_add} (measured; the paper assumes 20, 1, 1).
 * The dry-run counts replace the paper's estimate 10 c n log^2 V, whose
 * factor c it leaves open.  *mode: the first layer (layer 0) is Inter-CA
 * (the client encrypts its copies offline) unless its input, n ceil(F/t)
 * ciphertexts, exceeds max_inter_cts (0 = no limit); any other layer takes
 * the cheaper mode, ties to SpIntra-CA.  counts (may be NULL) = {R, T,
 * n ceil(F/t), ceil(log2 t)}.  FG_EINVAL / FG_ELEVEL as fg_plan_dry_run. */
#define FG_MODE_SPINTRA 0
#define FG_MODE_INTER 1
int fg_select_mode(const fg_params *params, const int32_t *row_ptr, const int32_t *col,
                   const double *val, int V, const double *W, int F, int Fp, const int32_t *perm,
                   const fg_plan_opts *opts, int layer, int n_copies, const double lat[3],
                   double max_inter_cts, int *mode, double cost[2], int64_t counts[4]);

/* Plan statistics for the learned planner (host only, like
 * fg_plan_dry_run): feat[FG_PLAN_FEATURES] = log2 V, log2 F, mean row
 * length of A-hat, log2(1 + max row length), log2 t, radix bits, mean bit
 * length of the node shifts |pi(u) - pi(v)| (AOO), groups, log2(1 +
 * rotations), log2(1 + masked terms), most lanes in a group, log2(1 + sum of
 * rotations x extended limbs), log2(1 + sum of terms x extended limbs),
 * log2(F (in_level + 1)), in_level. */
#define FG_PLAN_FEATURES 15
int fg_plan_features(const fg_params *params, const int32_t *row_ptr, const int32_t *col,
                     const double *val, int V, const double *W, int F, int Fp,
                     const int32_t *perm, const fg_plan_opts *opts, float *feat);
/* The same statistics of a plan already built (SpIntra-CA plans; the graph
 * it was built from is passed again as its CSR row_ptr, col). */
int fg_plan_features_built(const fg_plan *plan, const int32_t *row_ptr, const int32_t *col,
                           float *feat);

/* The learned planner's latency model (the paper's packing and ordering
 * choices, Sec. 3.2 and 3.4, made by a model instead of a search): a
 * three-layer perceptron y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 in FP32
 * on the GPU (current device), trained by full-batch Adam on the mean
 * squared error.  Parameters (host, float) are packed W1 [n_in][hidden],
 * b1 [hidden], W2 [hidden][hidden], b2 [hidden], W3 [hidden][1], b3 [1].
 * X is [n][n_in] row-major, y [n], all host memory.  fg_mlp_grad gives the
 * loss and its gradient in the packed order; fg_mlp_train runs `steps` Adam
 * steps (beta 0.9, 0.999, eps 1e-8) and writes the loss before each step
 * into losses (may be NULL).  fg_plan_choose scores n_cand feature rows and
 * returns the index of the lowest prediction.  Errors: FG_EINVAL, FG_ECUDA,
 * FG_EOOM; the message is fg_last_error(NULL). */
typedef struct fg_mlp fg_mlp;
int fg_mlp_create(int n_in, int hidden, const float *params, fg_mlp **out);
int fg_mlp_destroy(fg_mlp *mlp);
int fg_mlp_params(const fg_mlp *mlp, float *out);
int fg_mlp_forward(fg_mlp *mlp, const float *X, int n, float *y);
int fg_mlp_grad(fg_mlp *mlp, const float *X, const float *y, int n, float *loss, float *grad);
int fg_mlp_train(fg_mlp *mlp, const float *X, const float *y, int n, int steps, float lr,
                 float *losses);
int fg_plan_choose(fg_mlp *mlp, const float *features, int n_cand, float *pred, int *best);

/* Replace the encoding of mask `mask` by caller-given coefficients
 * [level+1][N] (host or device), e.g. an independent encoder's output. */
int fg_plan_set_plaintext(fg_plan *plan, int mask, const uint64_t *coeffs);

/* The layer (paper Sec. 3.2-3.3): in_cts = n_in packed ciphertexts at the
 * top level (fg_pack_features layout), out_cts = Fp ciphertexts [2][out_l+1][N]
 * holding A-hat X W column by column at the plan's node order (block 0 for
 * t > 1).  *out_level, *out_scale receive the output level and scale. */
int fg_gcn_layer_axw(fg_ctx *ctx, const fg_keys *keys, const fg_plan *plan,
                     const uint64_t *in_cts, int n_in, uint64_t *out_cts, int n_out,
                     int *out_level, double *out_scale);
/* The layer on seeded inputs (fg_pack_features_seeded): in_c0 = the n_in
 * c0 polynomials [n_in][L+1][N] (host or device) of seed's ciphertexts
 * 0..n_in-1.  Only c0 is copied from host memory (in column chunks that
 * overlap the combination, as for fg_gcn_layer_axw); the uniform parts are
 * regenerated on the device.  The outputs equal fg_gcn_layer_axw's on the
 * expanded ciphertexts (fg_expand_seeded) word for word.  FG_EINVAL for an
 * Inter-CA plan (its copies come from fg_pack_neighbor_copies). */
int fg_gcn_layer_axw_seeded(fg_ctx *ctx, const fg_keys *keys, const fg_plan *plan,
                            const uint64_t *in_c0, int n_in, uint64_t seed, uint64_t *out_cts,
                            int n_out, int *out_level, double *out_scale);

/* Batched layers (many queries, e.g. several graphs of one client, sharing
 * ctx and keys; the keys must hold every plan's rotations).  Query q runs
 * plans[q] on in_cts[q] (device, fg_pack_features layout) into out_cts[q]
 * (device, [Fp][2][out_l+1][N]); out_levels[q] receives its level (the scale
 * is ctx's Delta).  Up to opts->streams layers are in flight at once, each on
 * its own stream and workspace; opts->streams = 0 picks the count by timing
 * 8, 4, 2 and 1 on the first call (*streams_used, may be NULL, receives it).
 * With opts->graph = 1 the batch is captured into a CUDA graph on the first
 * call and replayed by later calls with the same plans and buffers.  With
 * opts->tune = 1 the first call also picks, by timing whole batch passes,
 * the launch configuration of the batch's kernels: the N = 2^16 NTT tile
 * (pass A columns and pass B rows per CTA, 16 or 8 each) and twiddle form
 * (held in registers per round, or loaded where used at one more CTA per
 * SM), the key switch's
 * register budget (its launch bound at the default or one CTA per SM
 * fewer) and the output count from which a group-MAC CTA runs three thread
 * groups (7, 4 or 13); fg_batch_tuning reports the choice.  Every
 * configuration computes the same words, and every query runs the kernels
 * of fg_gcn_layer_axw, so the outputs are the same word for word.  opts
 * NULL = {0, 1, 0}.  Host buffers: FG_EINVAL. */
typedef struct {
    int streams;   /* 1..16 layers in flight, 0 = chosen by timing */
    int graph;     /* 1 = capture once, replay while the arguments repeat */
    int tune;      /* 1 = choose the kernels' launch configuration by timing */
} fg_batch_opts;
int fg_gcn_layer_batch(fg_ctx *ctx, const fg_keys *keys, const fg_plan *const *plans, int n,
                       const uint64_t *const *in_cts, uint64_t *const *out_cts,
                       const fg_batch_opts *opts, int *out_levels, int *streams_used);
/* fg_gcn_layer_batch on seeded inputs (fg_pack_features_seeded): in_c0[q]
 * = query q's c0 parts [n_in][L+1][N] (device or page-locked host) of the
 * ciphertexts 0..n_in-1 of seed seeds[q]; the uniform parts are regenerated
 * on the device as in fg_gcn_layer_axw_seeded.  Same outputs, word for word,
 * as the queries run one at a time through fg_gcn_layer_axw_seeded.
 * FG_EINVAL for a null seeds array or an Inter-CA plan. */
int fg_gcn_layer_batch_seeded(fg_ctx *ctx, const fg_keys *keys, const fg_plan *const *plans, int n,
                              const uint64_t *const *in_c0, const uint64_t *seeds,
                              uint64_t *const *out_cts, const fg_batch_opts *opts, int *out_levels,
                              int *streams_used);
/* The batched form's launch configuration: cfg = {NTT pass-A columns, NTT
 * pass-B rows, NTT twiddles loaded where used (0/1), key-switch registers
 * (0 default, 1 one CTA per SM fewer, 2 keys in shared memory), key-switch column launches (1/2), fused ModUp
 * (0/1), fused ModDown (0/1), group-MAC three-group threshold, group-MAC
 * registers for three CTAs per SM (0/1), group-MAC products below 2^46 in
 * Karatsuba's form, three multiplies instead of four (1, the default, or 0)}; ms[0..*n) the
 * batch pass time of each configuration tried (the default first), at most
 * cap entries.  Before any tuned batch call cfg holds the context's
 * configuration and *n = 0. */
int fg_batch_tuning(const fg_ctx *ctx, int cfg[10], double *ms, int cap, int *n);
/* Fix the launch configuration every later call of this context uses
 * outside tuned batches (the same ten fields as fg_batch_tuning; NTT
 * tiles 16 or 8, key-switch registers 0 to 2, other flags 0 or 1, column
 * launches 1 or 2, group-MAC threshold >= 1).  Results do not change; speed may.  FG_EINVAL for other values. */
int fg_ctx_set_tuning(fg_ctx *ctx, const int cfg[10]);

/* Ciphertext products (paper Sec. 2.1 CMult; the x^2 activation between
 * GCN layers multiplies a ciphertext by itself): for each of n pairs,
 * out = Rescale((a0 b0, a0 b1 + a1 b0) + KS_relin(a1 b1)), with the
 * relinearisation key of fg_keygen (FG_EKEY without it).  a, b: [n][2][level+1][N]
 * coefficient domain (b may equal a); out: [n][2][level][N]; host or device.
 * The scale becomes scale_a * scale_b / q_level.  FG_ELEVEL for level < 1. */
int fg_mul_relin_rescale(fg_ctx *ctx, const fg_keys *keys, const uint64_t *a, const uint64_t *b,
                         int n, int level, uint64_t *out);

/* One rotation Rot(ct, k) (paper Sec. 2.1) with hybrid key switching,
 * ModUp taken before the automorphism (the hoisted order the layer uses).
 * ct, out: [2][level+1][N] (out may alias ct). */
int fg_rotate(fg_ctx *ctx, const fg_keys *keys, const uint64_t *ct, int level, int k,
              uint64_t *out);

/* Rescale by q_level (paper Sec. 2.1 and App. A: after a multiplication the
 * level drops by one), rounding each coefficient to the nearest integer:
 * out = floor((c + h) / q_l), h = (q_l - 1) / 2, i.e.
 * out_i = (c_i + [h]_{q_i} - [r]_{q_i}) q_l^-1 mod q_i with r = [c_l + h]_{q_l}
 * in [0, q_l).  Every key switch's ModDown uses the centred base conversion
 * (error of mean zero).  ct: [2][level+1][N], out: [2][level][N]. */
int fg_rescale(fg_ctx *ctx, const uint64_t *ct, int level, uint64_t *out);

/* Negacyclic product c = a * b mod (X^N + 1, q_i) for i <= level through the
 * device NTT (the ring product of paper Sec. 2.1).  [level+1][N] each. */
int fg_poly_mul(fg_ctx *ctx, const uint64_t *a, const uint64_t *b, int level, uint64_t *c);

/* The same product as fg_poly_mul, for callers that cannot allocate device
 * memory during the call: serving threads that must not block on or fail
 * in cudaMalloc (it can synchronise the device and run out of memory at any
 * time), and code whose device memory is owned and accounted by a host
 * framework or pool.  The paper has no counterpart; this is a deployment
 * aid.  a, b, c: DEVICE buffers [level+1][N] on the context's GPU (host
 * pointers and other GPUs' memory are rejected with FG_EINVAL); requires
 * (level+1) * N <= 2^18 words (FG_EINVAL otherwise).  Scratch comes from
 * one 4 MiB array compiled into the library, resident on every GPU that
 * loads it until the process exits; no cudaMalloc, cudaFree or other
 * allocating routine is called.  The first call for a context's GPU looks
 * up that array's device address on that GPU (make that first call before
 * any stream capture).  The call returns when c holds the product, like
 * fg_poly_mul.  Every call shares the array, so calls that overlap on the
 * GPU (other streams, other threads) race; nothing in it needs clearing,
 * since each call writes all the scratch it reads. */
int fg_poly_mul_noalloc(fg_ctx *ctx, const uint64_t *a, const uint64_t *b, int level,
                        uint64_t *c);

/* Forward (inverse = 0) or inverse NTT in place on DEVICE data
 * [count][N] whose limb c is taken modulo prime index prime_idx[c %
 * period] (0..n_q-1 for q_i, n_q.. for p_k).  The forward output order is
 * private to the library; inverse(forward(x)) = x.  For throughput
 * measurements. */
int fg_ntt(fg_ctx *ctx, uint64_t *data, int count, const int *prime_idx, int period,
           int inverse);

/* Measured integer-multiply throughput of the context's GPU (the ALU roof
 * of the modular kernels; the paper has no counterpart): eight independent
 * chains of one instruction per thread on eight 256-thread CTAs per SM,
 * timed with CUDA events.  op 0 = mad.wide.u32 (32 x 32 -> 64-bit product
 * plus a 64-bit addend), 1 = mul.hi.u32, 2 = mad.lo.u32, 3 = the pair
 * mad.lo.cc.u32 + madc.hi.u32 that adds a 32 x 32 -> 64-bit product to a
 * 64-bit sum (the step of the split products; the pair counts as one).
 * *ops_per_s: operations per second (one per thread) over the whole GPU.
 * FG_EINVAL for another op. */
int fg_int_mul_peak(fg_ctx *ctx, int op, double *ops_per_s);

#ifdef __cplusplus
}
#endif
#endif /* FICGCN_H */
