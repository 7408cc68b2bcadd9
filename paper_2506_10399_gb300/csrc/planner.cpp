// planner.cpp -- host planner of one encrypted GCN layer (FicGCN).
//
//  * latency-aware packing (paper Sec. 3.2, App. B.1): t = 1 when M <= V F';
//    otherwise the power of two t <= min(F, M/V) minimising
//    J(t; F, n) = 2 ceil(F n / t) + 20 ceil(log2 t), ties to the smaller t;
//  * combination constants round(W[f][j] q_l) (t = 1) or block-replicated W
//    masks plus the log t rotate-and-sum amounts B 2^i (t > 1);
//  * SpIntra-CA (Sec. 3.3): one token per edge v <- u (u != v) carrying
//    node u's value from slot perm[u] to slot perm[v]; the shift is taken
//    shortest-way round the ring (AOO, Sec. 3.3.2) and consumed r bits per
//    group from the low end (radix 2^r groups merge consecutive bit steps
//    into one rotation, the rotation merging of CPOO); in each group every
//    (lane, signed digit amount) is one rotation, tokens whose shift runs
//    out are removed into the accumulator with their weight A[v][u], moving
//    tokens that meet at one slot on the way to one destination are summed
//    from then on (each weighted in that step's mask; an extension of the
//    removal rule that keeps hubs' converging neighbours in one lane), and
//    the rest are placed first-fit into output lanes (a slot holds one
//    value per lane; a clash opens a new lane -- the paper's conflict;
//    filling the lowest lane first merges sparse lanes, CPOO's merging);
//  * the self weights A[v][v] multiply the column ciphertext in group 0.
// Every mask is applied at the group's level with scale q_level, so the
// rescale that closes the group keeps the ciphertext scale at Delta.
#include <algorithm>
#include <cmath>
#include <limits>
#include <map>
#include <unordered_map>

#include "fg_internal.h"

namespace planner {

static i64 packing_objective(i64 t, i64 F, i64 n)
{
    i64 pm = (F * n + t - 1) / t;
    i64 lg = 0;
    while ((1ll << lg) < t) lg++;
    return 2 * pm + 20 * lg;
}

int choose_t(int F, int n, int V, int Fp, int M)
{
    if ((i64)M <= (i64)V * Fp) return 1;
    int best = 1;
    i64 bj = packing_objective(1, F, n);
    for (int t = 2; t <= F && (i64)t * V <= M; t *= 2) {
        i64 j = packing_objective(t, F, n);
        if (j < bj) {
            bj = j;
            best = t;
        }
    }
    return best;
}

static int shift_amount(int src, int dst, int M, bool aoo)
{
    int r = ((src - dst) % M + M) % M;
    if (aoo && r > M / 2) r -= M;
    return r;
}

static int bitlen(i64 x)
{
    int b = 0;
    while (x) {
        b++;
        x >>= 1;
    }
    return b;
}

struct Token {
    int u, lane, pos, rho, dest;
    double w;
};

static void push_mask(fg_plan &pl, int level, std::vector<std::pair<int, double>> vals)
{
    std::sort(vals.begin(), vals.end());
    MaskC m;
    m.level = level;
    for (auto &sv : vals)
        if (sv.second != 0.0) {
            m.slots.push_back(sv.first);
            m.values.push_back(sv.second);
        }
    pl.masks.push_back(std::move(m));
}

void build(fg_plan &pl, const fg_ctx &ctx, const int32_t *row_ptr, const int32_t *col,
           const double *val, int V, const double *W, int F, int Fp, const int32_t *perm,
           const fg_plan_opts &o)
{
    const int M = ctx.slots;
    FG_CHECK(V >= 1 && F >= 1 && Fp >= 1, FG_EINVAL, "empty layer");
    FG_CHECK(row_ptr[0] == 0, FG_EINVAL, "row_ptr[0] must be 0");
    for (int v = 0; v < V; v++)
        FG_CHECK(row_ptr[v + 1] >= row_ptr[v], FG_EINVAL, "row_ptr must not decrease");
    const i64 nnz = row_ptr[V];
    for (i64 e = 0; e < nnz; e++)
        FG_CHECK(col[e] >= 0 && col[e] < V && std::isfinite(val[e]), FG_EINVAL, "bad A entry");
    for (i64 e = 0; e < (i64)F * Fp; e++) FG_CHECK(std::isfinite(W[e]), FG_EINVAL, "W not finite");

    int n = o.n_sampled;
    if (n <= 0) n = (int)std::llround((double)nnz / V);
    int t = o.t > 0 ? o.t : choose_t(F, n, V, Fp, M);
    FG_CHECK(t >= 1 && (t & (t - 1)) == 0 && t <= M, FG_EINVAL, "t must be a power of two");
    const int B = M / t;
    FG_CHECK((i64)V <= B, FG_EINVAL, "V nodes do not fit one block of M/t slots");
    std::vector<char> seen(B, 0);
    for (int v = 0; v < V; v++) {
        FG_CHECK(perm[v] >= 0 && perm[v] < B && !seen[perm[v]], FG_EINVAL,
                 "perm must be an injection of the nodes into [0, M/t)");
        seen[perm[v]] = 1;
    }
    pl.N = ctx.n;
    pl.M = M;
    pl.t = t;
    pl.B = B;
    pl.V = V;
    pl.F = F;
    pl.Fp = Fp;
    FG_CHECK(o.in_level >= 0 && o.in_level < ctx.nq, FG_ELEVEL, "input level out of range");
    pl.in_level = o.in_level > 0 ? o.in_level : ctx.nq - 1;
    pl.aoo = o.aoo ? 1 : 0;
    pl.perm.assign(perm, perm + V);

    // ---- combination
    const int l0 = pl.in_level;
    FG_CHECK(l0 >= 1, FG_ELEVEL, "the combination needs one level");
    if (t == 1) {
        const double ql = (double)ctx.primes[l0];
        pl.comb_consts.resize((size_t)F * Fp);
        for (i64 e = 0; e < (i64)F * Fp; e++) {
            double c = std::round(W[e] * ql);
            FG_CHECK(std::fabs(c) < 9.2e18, FG_EINVAL, "weight too large for the scale");
            pl.comb_consts[e] = (i64)c;
        }
    } else {
        const int nb = (F + t - 1) / t;
        pl.comb_masks.assign(nb, std::vector<int>(Fp));
        for (int b = 0; b < nb; b++)
            for (int j = 0; j < Fp; j++) {
                std::vector<std::pair<int, double>> vals;
                for (int k = 0; k < t; k++) {
                    int f = b * t + k;
                    if (f < F)
                        for (int s = 0; s < B; s++) vals.push_back({k * B + s, W[(size_t)f * Fp + j]});
                }
                push_mask(pl, l0, std::move(vals));
                pl.comb_masks[b][j] = (int)pl.masks.size() - 1;
            }
        for (int s = 1; s < t; s *= 2) pl.comb_rots.push_back(B * s);
    }

    // ---- tokens
    std::vector<double> self_w(V, 0.0);
    std::vector<Token> toks;
    for (int v = 0; v < V; v++)
        for (i64 e = row_ptr[v]; e < row_ptr[v + 1]; e++) {
            int u = col[e];
            if (u == v) {
                self_w[v] += val[e];
            } else {
                int rho = shift_amount(perm[u], perm[v], M, pl.aoo);
                toks.push_back({u, 0, perm[u], rho, perm[v], val[e]});
            }
        }
    i64 max_abs = 0;
    for (auto &tk : toks) max_abs = std::max<i64>(max_abs, std::llabs(tk.rho));
    const int total_bits = bitlen(max_abs);
    int level = l0 - 1;
    const int budget = level - o.min_out_level;
    int r = o.radix_bits;
    if (r <= 0) {
        r = 1;
        while (std::max(1, (total_bits + r - 1) / r) > budget && r < 30) r++;
    }
    const int G = std::max(1, (total_bits + r - 1) / r);
    FG_CHECK(level - G >= o.min_out_level && level - G >= 0, FG_ELEVEL,
             "level budget exhausted: " + std::to_string(G) + " groups from level " +
                 std::to_string(level));
    pl.radix_bits = r;

    int n_lanes = 1;
    pl.max_lanes = 1;
    int n_carriers = 0;
    for (int g = 0; g < G; g++) {
        const int lo = g * r;
        const int nb = std::max(0, std::min(r, total_bits - lo));
        // (src lane, k, dst) -> slot -> mask value; dst -1 = accumulator
        std::map<std::tuple<int, int, int>, std::map<int, double>> gterms;
        if (g == 0) {
            std::map<int, double> sv;
            for (int v = 0; v < V; v++)
                if (self_w[v] != 0.0) sv[perm[v]] = self_w[v];
            if (!sv.empty()) gterms[std::make_tuple(0, 0, -1)] = sv;
        }
        std::map<std::pair<int, int>, int> rot_set;   // (lane, k)
        struct Move {
            int tok, k, pos;
        };
        std::vector<Move> moving;
        for (size_t ti = 0; ti < toks.size(); ti++) {
            const Token &tk = toks[ti];
            const int digit = nb > 0 ? (int)((std::abs(tk.rho) >> lo) & ((1 << nb) - 1)) : 0;
            const int k = (digit << lo) * (tk.rho > 0 ? 1 : -1);
            const int newpos = ((tk.pos - k) % M + M) % M;
            if (k != 0) rot_set[{tk.lane, k}] = 1;
            if (tk.rho - k == 0) {   // arrival: removed into the accumulator
                FG_CHECK(newpos == tk.dest, FG_EINVAL, "planner: token missed its target");
                auto &m = gterms[std::make_tuple(tk.lane, k, -1)];
                FG_CHECK(!m.count(tk.dest), FG_EINVAL, "planner: repeated edge");
                m[tk.dest] = tk.w;
            } else {
                moving.push_back({(int)ti, k, newpos});
            }
        }
        // tokens meeting at one slot on the way to one destination are summed
        std::map<std::pair<int, int>, std::vector<int>> by_pd;   // (new slot, dest) -> moves
        for (size_t i = 0; i < moving.size(); i++)
            by_pd[{moving[i].pos, toks[moving[i].tok].dest}].push_back((int)i);
        std::map<std::tuple<int, int, int>, std::vector<int>> items;   // (lane, kmod, slot) -> moves
        std::vector<std::pair<std::pair<int, int>, std::vector<int>>> merged;
        for (auto &kv : by_pd) {
            if (kv.second.size() >= 2) {
                merged.push_back(kv);
            } else {
                const Move &mv = moving[kv.second[0]];
                items[std::make_tuple(toks[mv.tok].lane, ((mv.k % M) + M) % M, mv.pos)].push_back(
                    kv.second[0]);
            }
        }
        // per output lane, the content held at each slot (kEmpty: free);
        // content ids are node ids >= 0 or carrier ids < 0
        constexpr int kEmpty = std::numeric_limits<int>::min();
        std::vector<std::vector<int>> out_slots;
        auto place = [&](int p, int content, bool &joined) {
            for (size_t l = 0; l < out_slots.size(); l++)
                if (out_slots[l][p] == content) {
                    joined = true;
                    return (int)l;
                }
            joined = false;
            for (size_t l = 0; l < out_slots.size(); l++)
                if (out_slots[l][p] == kEmpty) {
                    out_slots[l][p] = content;
                    return (int)l;
                }
            out_slots.emplace_back(M, kEmpty);
            out_slots.back()[p] = content;
            return (int)out_slots.size() - 1;
        };
        std::vector<Token> nxt;
        for (auto &it : items) {   // ordered by (lane, k mod M, slot)
            const int p = std::get<2>(it.first);
            const Move &m0 = moving[it.second[0]];
            const int lane = toks[m0.tok].lane, k = m0.k, content = toks[m0.tok].u;
            bool joined;
            const int x = place(p, content, joined);
            if (!joined) gterms[std::make_tuple(lane, k, x)][p] = 1.0;
            for (int mi : it.second) {
                const Move &mv = moving[mi];
                Token t = toks[mv.tok];
                FG_CHECK(t.u == content, FG_EINVAL, "planner: two values share a lane slot");
                t.lane = x;
                t.pos = p;
                t.rho -= mv.k;
                nxt.push_back(t);
            }
        }
        for (auto &mg : merged) {   // ordered by (slot, dest)
            const int p = mg.first.first, d = mg.first.second;
            const int content = -(++n_carriers);
            bool joined;
            const int x = place(p, content, joined);
            const Move &m0 = moving[mg.second[0]];
            const int rho2 = toks[m0.tok].rho - m0.k;
            for (int mi : mg.second) {
                const Move &mv = moving[mi];
                const Token &t = toks[mv.tok];
                FG_CHECK(t.rho - mv.k == rho2, FG_EINVAL, "planner: carrier shift mismatch");
                auto &m = gterms[std::make_tuple(t.lane, mv.k, x)];
                FG_CHECK(!m.count(p), FG_EINVAL, "planner: carrier slot used twice");
                m[p] = t.w;
            }
            nxt.push_back({content, x, p, rho2, d, 1.0});
        }
        GroupC grp;
        grp.bit_lo = lo;
        grp.n_bits = nb;
        grp.level = level;
        grp.n_in = n_lanes;
        grp.n_out = (int)out_slots.size();
        for (auto &rk : rot_set) grp.rots.push_back(rk.first);
        auto kmod = [M](int k) { return ((k % M) + M) % M; };
        std::sort(grp.rots.begin(), grp.rots.end(),
                  [&](const std::pair<int, int> &a, const std::pair<int, int> &b) {
                      return a.first != b.first ? a.first < b.first : kmod(a.second) < kmod(b.second);
                  });
        std::vector<std::tuple<int, int, int>> tkeys;
        for (auto &kv : gterms) tkeys.push_back(kv.first);
        std::sort(tkeys.begin(), tkeys.end(), [&](const std::tuple<int, int, int> &a,
                                                  const std::tuple<int, int, int> &b) {
            if (std::get<0>(a) != std::get<0>(b)) return std::get<0>(a) < std::get<0>(b);
            if (kmod(std::get<1>(a)) != kmod(std::get<1>(b)))
                return kmod(std::get<1>(a)) < kmod(std::get<1>(b));
            return std::get<2>(a) < std::get<2>(b);
        });
        for (auto &tkey : tkeys) {
            std::vector<std::pair<int, double>> vals(gterms[tkey].begin(), gterms[tkey].end());
            push_mask(pl, level, std::move(vals));
            grp.terms.push_back({std::get<0>(tkey), std::get<1>(tkey), std::get<2>(tkey),
                                 (int)pl.masks.size() - 1});
        }
        pl.groups.push_back(std::move(grp));
        toks.swap(nxt);
        n_lanes = (int)out_slots.size();
        pl.max_lanes = std::max(pl.max_lanes, n_lanes);
        level--;
    }
    FG_CHECK(toks.empty(), FG_EINVAL, "planner: tokens left after the last group");
    pl.out_level = level;
}


void build_inter(fg_plan &pl, const fg_ctx &ctx, const int32_t *nbr, const double *wts, int V,
                 int n, const double *W, int F, int Fp, const int32_t *perm, const fg_plan_opts &o)
{
    const int M = ctx.slots;
    FG_CHECK(V >= 1 && n >= 1 && F >= 1 && Fp >= 1, FG_EINVAL, "empty layer");
    FG_CHECK(V <= M, FG_EINVAL, "V nodes do not fit the slots");
    std::vector<char> seen(M, 0);
    for (int v = 0; v < V; v++) {
        FG_CHECK(perm[v] >= 0 && perm[v] < M && !seen[perm[v]], FG_EINVAL,
                 "perm must be an injection of the nodes into [0, M)");
        seen[perm[v]] = 1;
        for (int k = 0; k < n; k++) {
            const int u = nbr[(size_t)v * n + k];
            FG_CHECK(u >= -1 && u < V && std::isfinite(wts[(size_t)v * n + k]), FG_EINVAL,
                     "bad neighbour entry");
        }
    }
    for (i64 e = 0; e < (i64)F * Fp; e++) FG_CHECK(std::isfinite(W[e]), FG_EINVAL, "W not finite");
    FG_CHECK(o.in_level >= 0 && o.in_level < ctx.nq, FG_ELEVEL, "input level out of range");
    pl.N = ctx.n;
    pl.M = M;
    pl.t = 1;
    pl.B = M;
    pl.V = V;
    pl.F = F;
    pl.Fp = Fp;
    pl.in_level = o.in_level > 0 ? o.in_level : ctx.nq - 1;
    pl.aoo = 1;
    pl.perm.assign(perm, perm + V);
    pl.n_copies = n;
    pl.radix_bits = -n;   // marks an Inter-CA plan in the records
    const int l0 = pl.in_level;
    FG_CHECK(l0 - 2 >= o.min_out_level && l0 >= 2, FG_ELEVEL, "Inter-CA needs two levels");
    const double ql = (double)ctx.primes[l0];
    pl.comb_consts.resize((size_t)F * Fp);
    for (i64 e = 0; e < (i64)F * Fp; e++) {
        double c = std::round(W[e] * ql);
        FG_CHECK(std::fabs(c) < 9.2e18, FG_EINVAL, "weight too large for the scale");
        pl.comb_consts[e] = (i64)c;
    }
    for (int k = 0; k < n; k++) {
        std::vector<std::pair<int, double>> vals;
        for (int v = 0; v < V; v++)
            if (nbr[(size_t)v * n + k] >= 0) vals.push_back({perm[v], wts[(size_t)v * n + k]});
        push_mask(pl, l0 - 1, std::move(vals));
    }
    pl.out_level = l0 - 2;
    pl.max_lanes = 1;
}

}  // namespace planner

namespace planner {

// Aggregation mode of one layer (paper Sec. 3.4, "Selecting Aggregation
// Mode"; App. B.2; Table 1's operation counts).  Both modes compute the
// combination Z = X W; they differ in how the n node arrangements of the
// aggregation are formed.  Per output column:
//   Inter-CA:   n ceil(F/t) PMult + Add (the combination of every copy),
//               n PMult + Add (the masked sum over the copies),
//               ceil(log2 t) Rot (the packing's rotate-and-sum);
//   SpIntra-CA: ceil(F/t) PMult + Add, ceil(log2 t) + R Rot, T PMult + Add,
//               with R rotations and T masked terms per column counted on
//               the plan itself (a dry run), which replaces the paper's
//               estimate 10 c n log^2 V and its unspecified factor c.
// Cost = sum of count x latency, latencies measured per operation (the
// paper assumes Rot = 20 PMult = 20 Add).  The first layer is Inter-CA (its
// copies are encrypted by the client, offline), unless the client's input,
// n ceil(F/t) ciphertexts, exceeds max_inter_cts; every other layer takes
// the cheaper mode (ties: SpIntra-CA).
void select_mode(const fg_plan &pl, int layer, int n_copies, const double lat[3], double max_inter_cts,
                 int *mode, double cost[2], int64_t counts[4])
{
    const double lr = lat[0], lp = lat[1], la = lat[2];
    const i64 F = pl.F, t = pl.t, n = n_copies;
    const i64 nb = (F + t - 1) / t;
    i64 lg = 0;
    while ((1ll << lg) < t) lg++;
    i64 R = 0, T = 0;
    for (const GroupC &g : pl.groups) {
        R += (i64)g.rots.size();
        T += (i64)g.terms.size();
    }
    const double inter = (double)(n * nb + n) * (lp + la) + (double)lg * lr;
    const double spintra = (double)(nb + T) * (lp + la) + (double)(lg + R) * lr;
    cost[0] = spintra;
    cost[1] = inter;
    counts[0] = R;
    counts[1] = T;
    counts[2] = n * nb;   // the client's Inter-CA input ciphertexts
    counts[3] = lg;
    const bool fits = max_inter_cts <= 0 || (double)(n * nb) <= max_inter_cts;
    if (layer == 0) *mode = fits ? FG_MODE_INTER : FG_MODE_SPINTRA;
    else *mode = (fits && inter < spintra) ? FG_MODE_INTER : FG_MODE_SPINTRA;
}

}  // namespace planner
