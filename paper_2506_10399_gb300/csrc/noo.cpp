// noo.cpp -- node order optimisation (Sec. 3.4, Alg. 1): the slot of every
// node, chosen so that SpIntra-CA needs few rotation steps.
//
// 1. Regions: breadth-first search from the highest-degree node not yet
//    placed (ties: lowest id), enqueueing siblings (nodes that share an
//    aggregation target) rather than neighbours, until the region holds TH
//    nodes or the queue runs empty.
// 2. Interleaving: the regions take turns, one slot each (ABCABC...), in
//    the order the search found them or, as an option, larger regions
//    first (the paper leaves the order open); a
//    region out of nodes gives its turn to a blank slot while any of the
//    M - V blanks remain, after that its turn is skipped.
// 3. Inside a region: the highest-degree node takes the region's first
//    slot; the others, in discovery order, take the free slot i with the
//    fewest conflicts k_n(i) = sum_j sum_rot Con_j^rot (Alg. 1) among the
//    nodes placed so far and n at i; ties go to the slot with the fewest
//    rotation steps to n's placed neighbours (set bits of the index
//    distances, one rotation per set bit), then to the lowest index.
//    Con_j^rot: within the region (positions 0..L-1) every edge v <- u
//    between placed nodes is a token carrying u's value from p(u) towards
//    p(v), shift d = p(u) - p(v) consumed bit by bit from the lowest; after
//    rotation rot it sits at p(u) - sign(d) (|d| mod 2^(rot+1)) unless it
//    has arrived (then it is removed); Con_j^rot = 1 when the tokens at j
//    after rotation rot carry two or more different values (a conflict of
//    Sec. 3.3).  The conflicts of the tokens already placed do not depend on
//    i, so only the change that n's own tokens bring is evaluated: per
//    rotation and position the first value seen and whether a second,
//    different one has been seen (tokens are only ever added).
#include <algorithm>
#include <deque>
#include <vector>

#include "fg_internal.h"

namespace {

struct Graph {
    std::vector<std::vector<int>> nb;   // off-diagonal entries of each row, ascending, unique
    std::vector<int> deg;
};

Graph neighbours(const int32_t *row_ptr, const int32_t *col, int V)
{
    Graph g;
    g.nb.resize(V);
    g.deg.resize(V);
    for (int v = 0; v < V; v++) {
        FG_CHECK(row_ptr[v + 1] >= row_ptr[v], FG_EINVAL, "row_ptr must not decrease");
        for (int e = row_ptr[v]; e < row_ptr[v + 1]; e++) {
            const int u = col[e];
            FG_CHECK(u >= 0 && u < V, FG_EINVAL, "column index out of range");
            if (u != v) g.nb[v].push_back(u);
        }
        std::sort(g.nb[v].begin(), g.nb[v].end());
        g.nb[v].erase(std::unique(g.nb[v].begin(), g.nb[v].end()), g.nb[v].end());
        g.deg[v] = (int)g.nb[v].size();
    }
    return g;
}

std::vector<std::vector<int>> regions_bfs(const Graph &g, int V, int TH)
{
    std::vector<int> order(V);
    for (int v = 0; v < V; v++) order[v] = v;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return g.deg[a] > g.deg[b]; });
    std::vector<char> placed(V, 0);
    std::vector<int> queued_in(V, -1);   // region that queued the node
    std::vector<std::vector<int>> regions;
    int oi = 0;
    for (;;) {
        while (oi < V && placed[order[oi]]) oi++;
        if (oi == V) break;
        const int r = (int)regions.size();
        regions.emplace_back();
        std::vector<int> &region = regions.back();
        std::deque<int> q{order[oi]};
        queued_in[order[oi]] = r;
        while (!q.empty() && (int)region.size() < TH) {
            const int u = q.front();
            q.pop_front();
            placed[u] = 1;
            region.push_back(u);
            for (int v : g.nb[u])
                for (int w : g.nb[v])
                    if (w != u && !placed[w] && queued_in[w] != r) {
                        queued_in[w] = r;
                        q.push_back(w);
                    }
        }
    }
    return regions;
}

std::vector<std::vector<int>> interleave(const std::vector<std::vector<int>> &regions, int V, int M)
{
    long long blanks = (long long)M - V;
    std::vector<int> left(regions.size());
    for (size_t r = 0; r < regions.size(); r++) left[r] = (int)regions[r].size();
    std::vector<std::vector<int>> slots(regions.size());
    int s = 0, remaining = V;
    while (remaining) {
        for (size_t r = 0; r < regions.size(); r++) {
            if (left[r]) {
                slots[r].push_back(s++);
                left[r]--;
                remaining--;
            } else if (blanks) {
                blanks--;
                s++;
            }
        }
    }
    return slots;
}

}  // namespace

extern "C" int fg_node_order_ex(const int32_t *row_ptr, const int32_t *col, int V, int M, int TH,
                                int region_order, int32_t *perm_out, int *n_regions)
{
    if (!row_ptr || !col || !perm_out || V < 1 || M < V || TH < 1 || region_order < 0 || region_order > 1)
        return FG_EINVAL;
    try {
        const Graph g = neighbours(row_ptr, col, V);
        auto regions = regions_bfs(g, V, TH);
        if (region_order == 1)   // larger regions take their turns first
            std::stable_sort(regions.begin(), regions.end(),
                             [](const std::vector<int> &a, const std::vector<int> &b) { return a.size() > b.size(); });
        const auto slots = interleave(regions, V, M);
        std::vector<int> idx(V, -1);   // slot index of a node within its region
        std::vector<int> region_of(V, -1);
        for (size_t r = 0; r < regions.size(); r++)
            for (int v : regions[r]) region_of[v] = (int)r;
        for (size_t r = 0; r < regions.size(); r++) {
            const std::vector<int> &region = regions[r];
            const int L = (int)region.size();
            int first = region[0];
            for (int v : region)
                if (g.deg[v] > g.deg[first] || (g.deg[v] == g.deg[first] && v < first)) first = v;
            std::vector<char> freed(L, 1);
            int B = 1;
            while ((1 << B) < L) B++;   // bit length of L - 1 (at least 1)
            std::vector<int> first_val((size_t)B * L, -1);
            std::vector<char> clash((size_t)B * L, 0);
            // the positions of a token from a to b after each rotation (until it arrives)
            struct Hit {
                int step, pos, val;
                bool operator<(const Hit &o) const
                {
                    return step != o.step ? step < o.step : pos != o.pos ? pos < o.pos : val < o.val;
                }
            };
            std::vector<Hit> hits;
            auto trace = [&](int a, int b, int val) {
                const int d = a - b, ad = std::abs(d);
                for (int st = 0; st < B; st++) {
                    const int done = ad & ((2 << st) - 1);
                    if (done == ad) break;   // arrived: removed
                    hits.push_back({st, d > 0 ? a - done : a + done, val});
                }
            };
            std::vector<int> placed_nb;
            auto tokens_of = [&](int n, int i) {
                hits.clear();
                for (int m : g.nb[n]) {
                    if (idx[m] < 0 || region_of[m] != (int)r) continue;
                    trace(idx[m], i, m);   // n aggregates m
                    trace(i, idx[m], n);   // m aggregates n
                }
            };
            idx[first] = 0;
            freed[0] = 0;
            for (int n : region) {
                if (n == first) continue;
                placed_nb.clear();
                for (int m : g.nb[n])
                    if (idx[m] >= 0 && region_of[m] == (int)r) placed_nb.push_back(idx[m]);
                int best = -1;
                long long best_con = 0, best_steps = 0;
                for (int i = 0; i < L; i++) {
                    if (!freed[i]) continue;
                    tokens_of(n, i);
                    std::sort(hits.begin(), hits.end());
                    long long con = 0;
                    for (size_t a = 0; a < hits.size();) {
                        size_t b = a;
                        while (b < hits.size() && hits[b].step == hits[a].step && hits[b].pos == hits[a].pos) b++;
                        const size_t cell = (size_t)hits[a].step * L + hits[a].pos;
                        if (!clash[cell]) {
                            const int f = first_val[cell];
                            bool c = false;
                            for (size_t k = a; k < b && !c; k++)
                                c = (f >= 0 && hits[k].val != f) || hits[k].val != hits[a].val;
                            con += c;
                        }
                        a = b;
                    }
                    long long steps = 0;
                    for (int j : placed_nb) steps += __builtin_popcount((unsigned)std::abs(i - j));
                    if (best < 0 || con < best_con || (con == best_con && steps < best_steps)) {
                        best = i;
                        best_con = con;
                        best_steps = steps;
                    }
                }
                idx[n] = best;
                freed[best] = 0;
                tokens_of(n, best);
                for (const Hit &h : hits) {
                    const size_t cell = (size_t)h.step * L + h.pos;
                    if (first_val[cell] < 0) first_val[cell] = h.val;
                    else if (first_val[cell] != h.val) clash[cell] = 1;
                }
            }
            for (int n : region) perm_out[n] = slots[r][idx[n]];
        }
        if (n_regions) *n_regions = (int)regions.size();
    } catch (const fg_error &e) {
        return e.code;
    } catch (const std::exception &) {
        return FG_EOOM;
    }
    return FG_OK;
}

extern "C" int fg_node_order(const int32_t *row_ptr, const int32_t *col, int V, int M, int TH,
                             int32_t *perm_out, int *n_regions)
{
    return fg_node_order_ex(row_ptr, col, V, M, TH, 0, perm_out, n_regions);
}
