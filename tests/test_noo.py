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


def test_greedy_slot_has_least_cost():
    """Brute force on a small graph: each node's slot index minimises the
    rotation-step cost among the slots free when it was placed."""
    w = wl.make_workload(graph="chung_lu", V=120, deg=4.0, gamma=2.5, F=4, Fp=2, seed=3)
    perm, nreg = noo.node_order(w.row_ptr, w.col, w.V, 256, TH=40)
    assert len(set(perm.tolist())) == w.V and perm.min() >= 0 and perm.max() < 256
    regions, nb, deg = noo.regions_bfs(w.row_ptr, w.col, w.V, 40)
    slots = noo.interleave(regions, w.V, 256)
    for region, sl in zip(regions, slots):
        idx = {v: sl.index(int(perm[v])) for v in region}
        first = min(region, key=lambda v: (-deg[v], v))
        assert idx[first] == 0
        taken = {0}
        placed = {first}
        for n in region:
            if n == first:
                continue
            pn = [idx[m] for m in nb[n] if m in placed]
            cost = lambda i: sum(bin(abs(i - j)).count("1") for j in pn)
            free = [i for i in range(len(region)) if i not in taken]
            best = min(free, key=lambda i: (cost(i), i))
            assert idx[n] == best
            taken.add(idx[n])
            placed.add(n)


@pytest.mark.parametrize("case", [("er", 64, 4.0, None, 128, 16), ("chung_lu", 300, 4.0, 2.5, 512, 48),
                                  ("chung_lu", 1000, 3.9, 2.2, 2048, 200)])
def test_library_node_order_matches_oracle(case):
    import paper_2506_10399_gb300 as fg
    graph, V, d, gamma, M, TH = case
    w = wl.make_workload(graph=graph, V=V, deg=d, gamma=gamma, F=4, Fp=2, seed=11)
    want, nr = noo.node_order(w.row_ptr, w.col, w.V, M, TH)
    got, nr2 = fg.node_order(w.row_ptr, w.col, M, TH)
    assert nr2 == nr
    np.testing.assert_array_equal(got, want)


def test_library_node_order_rejects_bad_input():
    import paper_2506_10399_gb300 as fg
    w = wl.make_workload(graph="er", V=16, deg=3.0, F=4, Fp=2, seed=0)
    with pytest.raises(fg.FicgcnError):
        fg.node_order(w.row_ptr, w.col, 8, 4)          # fewer slots than nodes
    bad = w.col.copy()
    bad[0] = 99
    with pytest.raises(fg.FicgcnError):
        fg.node_order(w.row_ptr, bad, 32, 4)
