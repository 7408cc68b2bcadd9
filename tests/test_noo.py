"""Node order optimisation (Sec. 3.4, Alg. 1): the oracle's stages against
their definitions, and the library's host implementation against the
oracle.  Parity of the heuristic itself is unpinned (no worked example in
the paper); what is pinned is that the order is a valid injection, that
each stage follows its rule, and that both implementations agree."""
import numpy as np
import pytest

from oracle import noo
from paper_2506_10399_gb300 import workloads as wl


def test_interleave_turns_and_blanks():
    """ABCABC...: exhausted regions take blanks while blanks remain, then are
    skipped (worked by hand)."""
    regions = [[0, 1, 2], [3], [4, 5]]
    assert noo.interleave(regions, 6, 9) == [[0, 3, 6], [1], [2, 5]]
    assert noo.interleave(regions, 6, 6) == [[0, 3, 5], [1], [2, 4]]


def test_interleave_one_blank_exact():
    # round 1: slots 0,1,2; round 2: r0 -> 3, r1 -> blank 4, r2 -> 5; round 3: r0 -> 6
    assert noo.interleave([[0, 1, 2], [3], [4, 5]], 6, 7) == [[0, 3, 6], [1], [2, 5]]


def _star_plus_path():
    # star 0-{1,2,3}, path 4-5-6, isolated 7
    edges = [(0, 1), (0, 2), (0, 3), (4, 5), (5, 6)]
    return wl.normalized_adjacency(8, np.array([a for a, b in edges]), np.array([b for a, b in edges]))


def test_regions_follow_sibling_bfs():
    """Seed = the highest degree (0, the star's centre).  The leaves 1, 2, 3
    share the target 0, so they are siblings of each other, while 0 has no
    sibling; regions end when their queue runs empty (worked by hand)."""
    rp, col, _ = _star_plus_path()
    regions, nb, deg = noo.regions_bfs(rp, col, 8, TH=8)
    assert deg[0] == 3 and deg[5] == 2
    # 0's targets are 1, 2, 3, whose rows hold only 0: no siblings -> region {0}
    assert regions[0] == [0]
    # next seed: node 5 (degree 2); targets 4, 6 hold only 5 -> region {5}
    assert regions[1] == [5]
    # then node 1 (degree 1, lowest id): target 0 holds 1, 2, 3 -> siblings 2, 3
    assert regions[2] == [1, 2, 3]
    assert regions[3] == [4, 6]
    assert regions[4] == [7]


def test_regions_respect_threshold():
    w = wl.config_workload("cora_like")
    regions, _, _ = noo.regions_bfs(w.row_ptr, w.col, w.V, TH=64)
    assert max(len(r) for r in regions) <= 64
    allv = sorted(v for r in regions for v in r)
    assert allv == list(range(w.V))


def count_conflicts(pos, nb, L):
    """Con summed over positions and rotations (Alg. 1), recomputed here by
    walking every token one rotation at a time: token v <- u starts at
    pos[u]; at rotation r, if bit r of |pos[u] - pos[v]| is set it moves
    2^r towards pos[v]; a token at pos[v] has arrived and leaves."""
    B = max(1, (L - 1).bit_length())
    toks = [(u, pos[u], pos[v]) for v in pos for u in nb[v] if u in pos]
    cur = [t[1] for t in toks]
    total = 0
    for r in range(B):
        cells = {}
        for k, (u, src, dst) in enumerate(toks):
            if cur[k] == dst:
                continue
            if (abs(src - dst) >> r) & 1:
                cur[k] += (1 << r) if dst > src else -(1 << r)
            if cur[k] != dst:
                cells.setdefault(cur[k], set()).add(u)
        total += sum(len(x) >= 2 for x in cells.values())
    return total


def test_conflict_count_hand_worked():
    """K4 on nodes 0..3, nodes 0, 2, 3 placed at indices 0, 1, 3 (L = 4, two
    rotations).  Tokens 2 <- 0 and 0 <- 2 arrive at rotation 0; 3 <- 0 moves
    0 -> 1, 0 <- 3 moves 3 -> 2, 3 <- 2 stays at 1 (bit 0 of |1 - 3| is 0),
    2 <- 3 stays at 3: after rotation 0 index 1 holds the values of 0 and 2,
    one conflict; after rotation 1 every token has arrived.  With node 3 at
    index 2 instead nothing collides."""
    nb = [[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]]
    assert noo.conflict_count({0: 0, 2: 1, 3: 3}, nb, 4) == 1
    assert noo.conflict_count({0: 0, 2: 1, 3: 2}, nb, 4) == 0
    assert count_conflicts({0: 0, 2: 1, 3: 3}, nb, 4) == 1


@pytest.mark.parametrize("seed", [3, 4])
def test_greedy_slot_has_least_conflicts(seed):
    """Brute force on a small graph: each node's slot index minimises the
    conflict count (then the rotation steps, then the index) among the
    slots free when it was placed."""
    w = wl.make_workload(graph="chung_lu", V=90, deg=4.0, gamma=2.5, F=4, Fp=2, seed=seed)
    perm, nreg = noo.node_order(w.row_ptr, w.col, w.V, 256, TH=30)
    assert len(set(perm.tolist())) == w.V and perm.min() >= 0 and perm.max() < 256
    regions, nb, deg = noo.regions_bfs(w.row_ptr, w.col, w.V, 30)
    slots = noo.interleave(regions, w.V, 256)
    collided = 0
    for region, sl in zip(regions, slots):
        L = len(region)
        idx = {v: sl.index(int(perm[v])) for v in region}
        first = min(region, key=lambda v: (-deg[v], v))
        assert idx[first] == 0
        pos = {first: 0}
        for n in region:
            if n == first:
                continue
            pn = [pos[m] for m in nb[n] if m in pos]
            free = [i for i in range(L) if i not in pos.values()]

            def key(i):
                return (count_conflicts({**pos, n: i}, nb, L),
                        sum(bin(abs(i - j)).count("1") for j in pn), i)
            best = min(free, key=key)
            assert idx[n] == best
            collided += key(best)[0] > 0
            pos[n] = idx[n]
    assert collided > 0      # the conflict term mattered somewhere


@pytest.mark.parametrize("case", [("er", 64, 4.0, None, 128, 16), ("chung_lu", 300, 4.0, 2.5, 512, 48),
                                  ("chung_lu", 400, 3.9, 2.2, 1024, 64)])
@pytest.mark.parametrize("region_order", [0, 1])
def test_library_node_order_matches_oracle(case, region_order):
    import paper_2506_10399_gb300 as fg
    graph, V, d, gamma, M, TH = case
    w = wl.make_workload(graph=graph, V=V, deg=d, gamma=gamma, F=4, Fp=2, seed=11)
    want, nr = noo.node_order(w.row_ptr, w.col, w.V, M, TH, region_order)
    got, nr2 = fg.node_order(w.row_ptr, w.col, M, TH, region_order)
    assert nr2 == nr
    np.testing.assert_array_equal(got, want)


def test_region_order_larger_first():
    """region_order 1: the interleaving turns go to larger regions first (the
    star-plus-path graph's regions have sizes 1, 1, 3, 2, 1)."""
    rp, col, _ = _star_plus_path()
    regions, _, _ = noo.regions_bfs(rp, col, 8, TH=8)
    ordered = sorted(regions, key=len, reverse=True)
    assert ordered[0] == [1, 2, 3] and ordered[1] == [4, 6]
    perm, _ = noo.node_order(rp, col, 8, 8, 8, region_order=1)
    assert perm[1] == 0 and perm[4] == 1       # first turns: regions {1,2,3}, {4,6}


def test_library_node_order_rejects_bad_input():
    import paper_2506_10399_gb300 as fg
    w = wl.make_workload(graph="er", V=16, deg=3.0, F=4, Fp=2, seed=0)
    with pytest.raises(fg.FicgcnError):
        fg.node_order(w.row_ptr, w.col, 8, 4)          # fewer slots than nodes
    bad = w.col.copy()
    bad[0] = 99
    with pytest.raises(fg.FicgcnError):
        fg.node_order(w.row_ptr, bad, 32, 4)


def test_planted_noo_slip_is_caught(monkeypatch):
    """A conflict counter that also counts cells holding a single value (a
    slip planted in the oracle) fails the hand-worked pin."""
    def loose(pos, nb, L):
        B = max(1, (L - 1).bit_length())
        total = 0
        for rot in range(B):
            at = set()
            for v, pv in pos.items():
                for u in nb[v]:
                    if u in pos:
                        d = pos[u] - pv
                        done = abs(d) % (1 << (rot + 1))
                        if done != abs(d):
                            at.add(pos[u] - (done if d > 0 else -done))
            total += len(at)
        return total
    monkeypatch.setattr(noo, "conflict_count", loose)
    with pytest.raises(AssertionError):
        test_conflict_count_hand_worked()
