"""Node order optimisation (NOO) of the oracle.  TEST INFRASTRUCTURE ONLY.

Written from the paper's Sec. 3.4 and Alg. 1: the node order pi (node ->
slot) is built in three stages.

1. Regions by a breadth-first search over siblings.  The seed is the node of
   highest degree among the nodes not yet placed (ties: lowest id); the
   search enqueues siblings instead of neighbours and stops when the region
   holds TH nodes or its queue runs empty.
2. Interleaved arrangement.  The regions take turns, one slot each, in
   region order (ABCABC...).  A region whose nodes are used up gives its turn
   to a blank slot while blanks (M - V of them) remain; after that its turn
   is skipped and the remaining regions alternate.
3. Conflict-least placement inside each region.  The region's slots are
   those stage 2 gave it.  Its highest-degree node takes the first slot; the
   others, in the order the search found them, each take the free slot i
   that minimises the total conflict count k_n(i) = sum_j sum_rot
   Con_j^rot (Alg. 1) of the nodes placed so far with n at i; among slots
   of equal count, the one with the fewest rotation steps to n's placed
   neighbours (the set bits of the index distances, one rotation per set
   bit, Sec. 3.3.1), then the lowest index.

Readings the paper leaves open (the library implements the same):
  * siblings of u: the nodes w != u with a common aggregation target v, i.e.
    u and w both in row v of A-hat (self loops ignored); enqueued in the
    order of v, then of w, both ascending;
  * degree: the number of off-diagonal entries of the row;
  * Con_j^rot (Alg. 1; a conflict is two different values meeting at one
    slot of one ciphertext, Sec. 3.3): within the region, positions are the
    slot indices 0..L-1; every edge v <- u between placed nodes is a token
    carrying u's value from p(u) to p(v), shift d = p(u) - p(v), moved bit
    by bit from the lowest (rotation rot moves it by sign(d) 2^rot when bit
    rot of |d| is set, so after rotation rot it sits at
    p(u) - sign(d) (|d| mod 2^(rot+1))), for rot = 0..bitlen(L-1)-1; a token
    that has reached p(v) is removed (it has arrived, Sec. 3.3); Con_j^rot
    is 1 when, after rotation rot, the tokens at position j carry two or
    more different values.

Parity unpinned: NOO is a heuristic with no worked example in the paper.
Its output is pinned only as a valid injection of the nodes into the slots,
and the library's implementation is compared with this one.
"""
from collections import deque

import numpy as np


def _neighbours(row_ptr, col, V):
    nb = []
    for v in range(V):
        r = [int(u) for u in col[row_ptr[v]:row_ptr[v + 1]] if int(u) != v]
        nb.append(sorted(set(r)))
    return nb


def regions_bfs(row_ptr, col, V, TH):
    """Stage 1: list of regions, each a list of nodes in discovery order."""
    nb = _neighbours(row_ptr, col, V)
    deg = [len(n) for n in nb]
    order = sorted(range(V), key=lambda v: (-deg[v], v))
    placed = [False] * V
    regions = []
    oi = 0
    while True:
        while oi < V and placed[order[oi]]:
            oi += 1
        if oi == V:
            break
        seed = order[oi]
        region = []
        queued = {seed}
        q = deque([seed])
        while q and len(region) < TH:
            u = q.popleft()
            placed[u] = True
            region.append(u)
            for v in nb[u]:
                for w in nb[v]:
                    if w != u and not placed[w] and w not in queued:
                        queued.add(w)
                        q.append(w)
        regions.append(region)
    return regions, nb, deg


def interleave(regions, V, M):
    """Stage 2: the slots of each region, in slot order."""
    blanks = M - V
    if blanks < 0:
        raise ValueError("more nodes than slots")
    left = [len(r) for r in regions]
    slots = [[] for _ in regions]
    s = 0
    remaining = V
    while remaining:
        for r in range(len(regions)):
            if left[r]:
                slots[r].append(s)
                left[r] -= 1
                remaining -= 1
                s += 1
            elif blanks:
                blanks -= 1
                s += 1
    return slots


def conflict_count(pos, nb, L):
    """sum_j sum_rot Con_j^rot for the nodes placed at pos (node -> index):
    the tokens of every edge v <- u with both ends placed, simulated bit by
    bit (see the module docstring)."""
    B = max(1, (L - 1).bit_length())
    total = 0
    for rot in range(B):
        at = {}
        for v, pv in pos.items():
            for u in nb[v]:
                if u not in pos:
                    continue
                d = pos[u] - pv
                done = abs(d) % (1 << (rot + 1))
                if done == abs(d):
                    continue                     # arrived: removed
                p = pos[u] - (done if d > 0 else -done)
                at.setdefault(p, set()).add(u)
        total += sum(1 for vals in at.values() if len(vals) >= 2)
    return total


def node_order(row_ptr, col, V, M, TH, region_order=0):
    """pi as an int64 array: node -> slot in [0, M).  region_order 0: the
    regions take their interleaving turns in the order the search found
    them; 1: larger regions first, ties in search order (the paper leaves
    the order open)."""
    regions, nb, deg = regions_bfs(row_ptr, col, V, TH)
    if region_order == 1:
        regions = sorted(regions, key=len, reverse=True)   # stable: ties keep search order
    slots = interleave(regions, V, M)
    perm = np.full(V, -1, dtype=np.int64)
    for region, sl in zip(regions, slots):
        L = len(region)
        first = min(region, key=lambda v: (-deg[v], v))
        idx = {first: 0}              # node -> slot index within the region
        free = [True] * L
        free[0] = False
        for n in region:
            if n == first:
                continue
            placed_nb = [idx[m] for m in nb[n] if m in idx]
            best, best_i = None, None
            for i in range(L):
                if not free[i]:
                    continue
                idx[n] = i
                cost = (conflict_count(idx, nb, L), sum(bin(abs(i - j)).count("1") for j in placed_nb))
                if best is None or cost < best:
                    best, best_i = cost, i
            idx[n] = best_i
            free[best_i] = False
        for n, i in idx.items():
            perm[n] = sl[i]
    return perm, len(regions)
