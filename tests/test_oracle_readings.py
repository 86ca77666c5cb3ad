"""Hand-worked pins of the oracle's readings of the paper's open choices.

The invariants in test_oracle.py (connected patches, the cap, valid and
minimal separators) hold for any choice of seed, split or release order, so
they cannot tell a right reading from a wrong one. Each case below is small
enough to work out by hand from the rule alone; the expected values are
written out with their derivation, never taken from the oracle.

Readings pinned here (the determinism contract):
  R4  Lloyd re-centring: the new seed is the patch vertex of maximum hop depth
      from the patch boundary, ties to the lowest id; a patch without boundary
      keeps its seed (Section 4.1 step 1; RXMesh's Lloyd patcher in the paper).
  R5  cap split: the second seed is the vertex farthest from the seed inside
      the patch, ties to the lowest id; new ranks follow all existing ranks in
      the order of the parent rank.
  R8  bipartition (Algorithm 2 step 2): components by smallest patch id;
      r0 = min (degree, id); r1 = min (degree, id) on the last BFS level from
      r0; order by (BFS level from r1, id); Left = the prefix that best halves
      the remaining vertex weight (ties to the shorter prefix), kept within
      the patch capacity of each child's subtree.
  R9  refinement (Algorithm 2 step 4): superset vertices are released in
      increasing (crossing degree, tie hash, id), a vertex being released iff
      none of its crossing neighbours was released before it.
"""
from __future__ import annotations

import numpy as np

import oracle as O

M64 = (1 << 64) - 1


def graph(n: int, edges) -> O.Graph:
    """Symmetric CSR of an undirected edge list (rows sorted)."""
    nb = [set() for _ in range(n)]
    for a, b in edges:
        nb[a].add(b)
        nb[b].add(a)
    rp = np.zeros(n + 1, np.int32)
    col = []
    for v in range(n):
        col += sorted(nb[v])
        rp[v + 1] = len(col)
    return O.Graph(rp, np.array(col, np.int32))


def path(n: int) -> O.Graph:
    return graph(n, [(i, i + 1) for i in range(n - 1)])


def tie_hash(v: int) -> int:
    """High 32 bits of SplitMix64's output for state v (Steele, Lea & Flood
    2014), restated from the published generator; test_oracle.py checks the
    oracle's generator against the published output sequence."""
    z = (v + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return (z ^ (z >> 31)) >> 32


# ---- R4 Lloyd ------------------------------------------------------------------

# The tree 0-1-2-3-4 with the branch 2-5-6-7, seeds [2, 7].
#   First labelling: hop distances from 2 and from 7 give patch 0 = {0..5}
#   (5 is 1 from 2, 2 from 7) and patch 1 = {6, 7}.
#   Lloyd round 1: the boundary is {5, 6}. Depths inside patch 0 from 5:
#   2 -> 1, 1 and 3 -> 2, 0 and 4 -> 3; maximum 3, tied between 0 and 4 ->
#   the lower id, 0. Patch 1 from 6: 7 -> 1, so 7. Seeds [0, 7].
#   Relabel: 5 is 3 from 0 and 2 from 7 -> patch 1; 0..4 stay in patch 0.
#   Round 2: boundary {2, 5}; depths in {0..4} from 2: 0 and 4 at 2 -> 0 again;
#   in {5, 6, 7} from 5: 7 at 2 -> 7. Nothing changes.
LLOYD_TREE = [(0, 1), (1, 2), (2, 3), (3, 4), (2, 5), (5, 6), (6, 7)]


def test_lloyd_no_rounds_keeps_first_labelling():
    lab, seeds, k = O.patches_from_seeds(graph(8, LLOYD_TREE), [2, 7], cap=100, lloyd_rounds=0)
    assert k == 2
    assert seeds.tolist() == [2, 7]
    assert lab.tolist() == [0, 0, 0, 0, 0, 0, 1, 1]


def test_lloyd_moves_seed_to_deepest_vertex_lowest_id():
    for rounds in (1, 2):
        lab, seeds, k = O.patches_from_seeds(graph(8, LLOYD_TREE), [2, 7], cap=100, lloyd_rounds=rounds)
        # minimum depth would give [5, 6]; ties to the highest id [4, 7]
        assert seeds.tolist() == [0, 7], rounds
        assert lab.tolist() == [0, 0, 0, 0, 0, 1, 1, 1], rounds


def test_lloyd_patch_without_boundary_keeps_its_seed():
    # one seed on a path: the only patch has no boundary vertex
    lab, seeds, k = O.patches_from_seeds(path(7), [3], cap=100, lloyd_rounds=2)
    assert (k, seeds.tolist(), lab.tolist()) == (1, [3], [0] * 7)


def test_lloyd_traced_rounds_on_a_mesh_follow_the_rule():
    """On a real mesh every traced Lloyd seed is a vertex of maximum depth
    from its patch boundary (lowest id among them), depths recomputed here by
    a plain BFS per patch."""
    import meshgen
    m = meshgen.grid64(3)
    g = O.graph_from_faces(m.faces, m.n)
    t = O.order_trace(g, 256, seed=3, lloyd_rounds=2)
    for r in range(2):
        lab = t.labels[r]
        k = int(lab.max()) + 1
        depth = np.full(g.n, -1)
        front = [v for v in range(g.n) if any(lab[u] != lab[v] for u in g.neighbors(v))]
        for v in front:
            depth[v] = 0
        while front:
            nxt = []
            for v in front:
                for u in g.neighbors(v):
                    if lab[u] == lab[v] and depth[u] < 0:
                        depth[u] = depth[v] + 1
                        nxt.append(u)
            front = nxt
        want = []
        for p in range(k):
            mem = np.flatnonzero(lab == p)
            if depth[mem].max() < 0:
                want.append(int(t.seeds0[p]) if r == 0 else int(t.lloyd_seeds[r - 1][p]))
                continue
            d = depth[mem].max()
            want.append(int(mem[depth[mem] == d].min()))
        assert t.lloyd_seeds[r].tolist() == want, r


# ---- R5 cap split ----------------------------------------------------------------

def test_cap_split_farthest_vertex_lowest_id():
    # Path 0..6, seed 3, cap 4.
    #   Split 1: patch 0 has 7 > 4 vertices; farthest from 3 are 0 and 6 (3
    #   hops) -> 0, rank 1. Relabel from 3 (rank 0) and 0 (rank 1): 0, 1 go to
    #   rank 1 (1 is 1 hop from 0, 2 from 3); 2..6 stay in rank 0.
    #   Split 2: rank 0 = {2..6} has 5 > 4; farthest from 3 inside it is 6 ->
    #   rank 2. Relabel: 5, 6 -> rank 2 (5 is 1 from 6, 2 from 3).
    # Ties to the highest id would start with 6 and end with labels
    # [2, 2, 0, 0, 0, 1, 1].
    lab, seeds, k = O.patches_from_seeds(path(7), [3], cap=4, lloyd_rounds=0)
    assert k == 3
    assert seeds.tolist() == [3, 0, 6]
    assert lab.tolist() == [1, 1, 0, 0, 0, 2, 2]


def test_cap_split_ranks_follow_parent_rank():
    # Path 0..13, seeds 3 and 10, cap 4: patches {0..6} and {7..13} (6 is 3
    # from 3 and 4 from 10). Both split in the same round, in increasing
    # parent rank: rank 2 = 0 (farthest from 3, tie with 6 -> 0), rank 3 = 7
    # (farthest from 10, tie with 13 -> 7). After relabelling, {2..6} and
    # {9..13} still hold 5 > 4 vertices: rank 4 = 6 (from 3), rank 5 = 13
    # (from 10). Final: {0,1} 2, {2,3,4} 0, {5,6} 4, {7,8} 3, {9,10,11} 1,
    # {12,13} 5.
    lab, seeds, k = O.patches_from_seeds(path(14), [3, 10], cap=4, lloyd_rounds=0)
    assert k == 6
    assert seeds.tolist() == [3, 10, 0, 7, 6, 13]
    assert lab.tolist() == [2, 2, 0, 0, 0, 4, 4, 3, 3, 1, 1, 1, 5, 5]


# ---- R8 bipartition ----------------------------------------------------------------

def root_sides(g, groups, k):
    t = O.order_trace(g, given=np.asarray(groups, np.int32), k=k)
    return t.side_at[0].tolist(), t


def test_bisection_splits_by_weight_not_count():
    # Groups on the path 0..7: A = {0} (w 1), B = {1..5} (w 5), C = {6, 7}
    # (w 2); quotient path A-B-C, k = 3, D = 2, child capacity c = 2 at the
    # root, so j in [1, 2]. r0 = A (degree 1, id 0); the last level from A is
    # {C}, r1 = C; order C, B, A. W = 8: P_1 = 2 (|4 - 8| = 4), P_2 = 7
    # (|14 - 8| = 6) -> Left = {C}. Halving the count (ceil) would also put B
    # on the left.
    sides, _ = root_sides(path(8), [0, 1, 1, 1, 1, 1, 2, 2], 3)
    assert sides == [1, 1, 0]


def test_bisection_weight_prefers_longer_prefix_when_closer():
    # A = {0..4} (w 5), B = {5} (w 1), C = {6, 7} (w 2) on the path 0..7:
    # order C, B, A; W = 8: P_1 = 2 (4), P_2 = 3 (2) -> Left = {C, B}.
    # Halving the count (floor) would give Left = {C}.
    sides, _ = root_sides(path(8), [0, 0, 0, 0, 0, 1, 2, 2], 3)
    assert sides == [1, 0, 0]


def test_bisection_weight_tie_goes_to_shorter_prefix():
    # three groups of two on the path 0..5: order C, B, A; W = 6: P_1 = 2 and
    # P_2 = 4 are both 2 from the half -> the shorter prefix, Left = {C}.
    sides, _ = root_sides(path(6), [0, 0, 1, 1, 2, 2], 3)
    assert sides == [1, 1, 0]


def test_bisection_respects_subtree_capacity():
    # A = {0..9} (w 10), B = {10}, C = {11}, D = {12} on the path 0..12:
    # quotient path A-B-C-D, k = 4, D = 2, so each child of the root holds at
    # most c = 2 patches: j in [2, 2]. r0 = A, r1 = D, order D, C, B, A with
    # weights 1, 1, 1, 10; unconstrained the best cut would be j = 3
    # (|6 - 13| = 7), which would leave three patches below one child.
    sides, t = root_sides(path(13), [0] * 10 + [1, 2, 3], 4)
    assert sides == [1, 1, 0, 0]
    # and every leaf is then a single patch
    o = t.ordering
    for node in range(len(o.node_size)):
        blk = o.perm[o.node_begin[node]:o.node_begin[node] + o.node_size[node]]
        if blk.size and 2 * node + 1 >= len(o.node_size):
            assert np.unique(np.asarray([0] * 10 + [1, 2, 3])[blk]).size == 1


def test_bisection_second_root_is_min_degree_then_id_on_last_level():
    # Single-vertex patches (the quotient graph is G itself) on the edges
    # 0-1, 1-2, 1-3, 1-4, 2-4. Degrees 1, 4, 2, 1, 2; r0 = 0. Levels from 0:
    # {0}, {1}, {2, 3, 4}; on the last level (degree, id) = (2,2), (1,3), (2,4)
    # -> r1 = 3. Order from 3: 3 | 1 | 0 2 4. k = 5, D = 3, c = 4, j in [1, 4];
    # W = 5: j = 2 and 3 both leave 1 -> j = 2, Left = {3, 1}.
    # r1 = highest id (4) would order 4 | 1 2 | 0 3, r1 = lowest id (2) 2 | 1 4
    # | 0 3: Left {4, 1} or {2, 1}.
    g = graph(5, [(0, 1), (1, 2), (1, 3), (1, 4), (2, 4)])
    sides, _ = root_sides(g, list(range(5)), 5)
    assert sides == [1, 0, 1, 0, 1]


def test_bisection_orders_each_level_by_id():
    # A star: centre 0, leaves 1..6 (single-vertex patches). r0 = 1 (degree 1,
    # lowest id); the last level from 1 is {2..6}, all of degree 1 -> r1 = 2.
    # Order from 2: 2 | 0 | 1 3 4 5 6. k = 7, D = 3, c = 4, j in [3, 4];
    # W = 7: j = 3 and 4 tie -> 3, Left = {2, 0, 1}: the first vertex of the
    # last level by id. Decreasing ids within a level would take 6 instead.
    g = graph(7, [(0, i) for i in range(1, 7)])
    sides, _ = root_sides(g, list(range(7)), 7)
    assert sides == [0, 0, 0, 1, 1, 1, 1]


def test_bisection_orders_components_by_smallest_id():
    # Edges 0-5, 2-3, 3-4 and the isolated vertex 1 (single-vertex patches).
    # Components by smallest id: {0, 5}, {1}, {2, 3, 4}. {0, 5}: r0 = 0,
    # r1 = 5, order 5 0; {1}: 1; {2, 3, 4}: r0 = 2, r1 = 4, order 4 3 2.
    # Order 5 0 1 4 3 2; k = 6, D = 3, c = 4, j in [2, 4]; W = 6 -> j = 3,
    # Left = {5, 0, 1}. Largest component first would give Left = {4, 3, 2}.
    g = graph(6, [(0, 5), (2, 3), (3, 4)])
    sides, _ = root_sides(g, list(range(6)), 6)
    assert sides == [0, 0, 1, 1, 1, 0]


# ---- R9 refinement ----------------------------------------------------------------

def test_refinement_releases_low_crossing_degree_first():
    # Triangle 0-1-2 with groups A = {0}, B = {1, 2}: k = 2, D = 1, order B, A
    # (r0 = A, r1 = B), so B is left and A right. Crossing edges 0-1 and 0-2:
    # crossing degrees 2, 1, 1. In increasing order 1 and 2 are released first
    # (0 is not yet released), then 0 has released crossing neighbours and
    # stays: separator {0}, and 1, 2 go to the left child. Releasing in
    # decreasing order would release 0 and keep {1, 2}.
    g = graph(3, [(0, 1), (0, 2), (1, 2)])
    t = O.order_trace(g, given=np.array([0, 1, 1], np.int32), k=2)
    assert t.ordering.node_of.tolist() == [0, 1, 1]


def test_refinement_breaks_crossing_degree_ties_by_hash():
    # The edge 0-1 with single-vertex patches: order 1, 0 (r0 = 0, r1 = 1), so
    # 1 is left and 0 right; both have crossing degree 1. The tie key is the
    # SplitMix64 hash: the vertex with the smaller hash is released, the other
    # is the separator. By id, 0 would be released.
    assert tie_hash(1) < tie_hash(0)        # 0x910a2dec < 0xe220a839
    t = O.order_trace(path(2), given=np.array([0, 1], np.int32), k=2)
    assert t.ordering.node_of.tolist() == [0, 1]


def test_refinement_hash_order_on_a_longer_cut():
    # Groups A = {0, 1, 2}, B = {3, 4, 5} on the ladder 0-1-2 / 3-4-5 with
    # rungs 0-3, 1-4, 2-5: k = 2, order B, A (r0 = A, r1 = B): B left, A right.
    # Every vertex has crossing degree 1; each rung keeps exactly one end, the
    # one released later, i.e. the one with the larger hash:
    # rung 0-3: hashes 0xe220a839 vs 0x1d0b14e4 -> 3 released, 0 separator;
    # rung 1-4: 0x910a2dec vs 0x6e73e372 -> 4 released, 1 separator;
    # rung 2-5: 0x975835de vs 0x63033b0c -> 5 released, 2 separator.
    # So A = {0, 1, 2} is the separator (node 0) and B goes to node 1.
    g = graph(6, [(0, 1), (1, 2), (3, 4), (4, 5), (0, 3), (1, 4), (2, 5)])
    for a, b in ((0, 3), (1, 4), (2, 5)):
        assert tie_hash(b) < tie_hash(a)
    t = O.order_trace(g, given=np.array([0, 0, 0, 1, 1, 1], np.int32), k=2)
    assert t.ordering.node_of.tolist() == [0, 0, 0, 1, 1, 1]
