"""Pins of the CPU oracle against things other than itself: published test
vectors, closed forms, brute force on tiny inputs, textbook special cases and
the invariants the paper states for nested dissection."""
import numpy as np
import pytest

import meshgen as M
import oracle as O
from brute import (adj_lists, bfs_from, connected, elimination_game, fill_of_order,
                   min_fill_exhaustive, voronoi_brute)


def _faces_graph(mesh):
    return O.graph_from_faces(mesh.faces, mesh.n)


def _graph_from_edges(n, edges):
    rows = [[] for _ in range(n)]
    for a, b in edges:
        rows[a].append(b); rows[b].append(a)
    rp = np.zeros(n + 1, np.int32); col = []
    for i, r in enumerate(rows):
        r = sorted(set(r)); col += r; rp[i + 1] = len(col)
    return O.Graph(rp, np.array(col, np.int32))


# --- contract R1: the published SplitMix64 sequence --------------------------

def test_splitmix64_published_vector():
    # Reference outputs of SplitMix64 started from state 1234567 (Steele, Lea &
    # Flood 2014; the sequence printed by Vigna's reference splitmix64.c).
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    # seed_hash(seed, v) is the generator at state seed*gamma + v, i.e. the
    # (seed+1)-th output of the stream started at state v.
    assert [O.seed_hash(k, 1234567) for k in range(5)] == want


def test_seed_rule_counts():
    n = 100000
    for cap in (64, 256, 512):
        kt = -(-2 * n // cap)
        c = O.seeds(n, cap, 7).size
        assert abs(c - kt) < 6 * np.sqrt(kt), (cap, c, kt)
    # cap 1 or 2 => k_target >= n => every vertex is a seed
    assert O.seeds(50, 1, 3).size == 50
    assert O.seeds(50, 2, 3).size == 50
    s = O.seeds(1000, 100, 5)
    assert np.all(np.diff(s) > 0)


# --- Section 2: G is the graph of A without diagonal -------------------------

def test_graph_closed_forms():
    g = _faces_graph(M.grid64(0))
    E = g.col.size // 2
    assert (g.n, E) == (4096, 12033)
    assert g.n - E + 7938 == 1                     # disc: Euler characteristic 1
    for lvl in range(6):
        m = M.icosphere(lvl)
        g = _faces_graph(m)
        E = g.col.size // 2
        assert E == 30 * 4 ** lvl
        assert m.n - E + m.n_faces == 2            # sphere
    for s in range(3):
        m = M.torus(17, 13, 0.3, s)
        g = _faces_graph(m)
        assert g.col.size // 2 == 3 * m.n
        assert m.n - 3 * m.n + m.n_faces == 0      # torus
    g = _faces_graph(M.icosphere7(0))
    assert (g.n, g.col.size) == (163842, 983040)
    # symmetric, sorted, no diagonal
    for v in range(0, g.n, 997):
        nb = g.neighbors(v)
        assert np.all(np.diff(nb) > 0) and v not in nb
        for u in nb:
            assert v in g.neighbors(u)


def test_graph_degenerate_faces_and_errors():
    f = np.array([[0, 1, 1], [2, 2, 2], [0, 1, 3]], np.int32)
    g = O.graph_from_faces(f, 5)
    assert adj_lists(g) == [[1, 3], [0, 3], [], [0, 1], []]
    with pytest.raises(ValueError):
        O.graph_from_faces(np.array([[0, 1, 5]], np.int32), 5)


def test_graph_from_pattern_scalar_and_block():
    m = M.torus(6, 5, 0.3, 2)
    g = _faces_graph(m)
    n = g.n
    # scalar pattern = G + I
    rows = [sorted(set(g.neighbors(v).tolist()) | {v}) for v in range(n)]
    rp = np.cumsum([0] + [len(r) for r in rows]).astype(np.int32)
    col = np.array(sum(rows, []), np.int32)
    g1 = O.graph_from_pattern(rp, col, 1)
    assert np.array_equal(g1.rowptr, g.rowptr) and np.array_equal(g1.col, g.col)
    # 3x3 dense blocks (Section 6.5): compress back to the vertex graph
    b = 3
    drows = []
    for i in range(n * b):
        v = i // b
        drows.append(sorted(b * u + c for u in rows[v] for c in range(b)))
    drp = np.cumsum([0] + [len(r) for r in drows]).astype(np.int32)
    dcol = np.array(sum(drows, []), np.int32)
    g3 = O.graph_from_pattern(drp, dcol, 3)
    assert np.array_equal(g3.rowptr, g.rowptr) and np.array_equal(g3.col, g.col)
    # a one-sided entry is rejected
    bad_rp = np.array([0, 1, 1], np.int32); bad_col = np.array([1], np.int32)
    with pytest.raises(ValueError):
        O.graph_from_pattern(bad_rp, bad_col, 1)


# --- contract R2: Voronoi labelling vs one BFS per source ---------------------

@pytest.mark.parametrize("seed", range(6))
def test_voronoi_matches_bruteforce(seed):
    rng = np.random.default_rng(seed)
    mesh = [M.shuffle(M.torus(9, 7, 0.3, seed), seed), M.shuffle(M.grid(10, 9), seed),
            M.shuffle(M.icosphere(2), seed)][seed % 3]
    g = _faces_graph(mesh)
    adj = adj_lists(g)
    ns = int(rng.integers(1, 12))
    src = rng.choice(g.n, ns, replace=False)
    rank = rng.permutation(ns)
    d, l = O.voronoi(g, src, rank)
    bd, bl = voronoi_brute(adj, src, rank)
    assert np.array_equal(d, bd) and np.array_equal(l, bl)
    group = rng.integers(0, 3, g.n)
    d, l = O.voronoi(g, src, rank, group)
    bd, bl = voronoi_brute(adj, src, rank, group)
    assert np.array_equal(d, bd) and np.array_equal(l, bl)


# --- contract R1-R5: patching invariants --------------------------------------

def _disconnected_mesh():
    a = M.shuffle(M.torus(12, 10, 0.3, 1), 1)
    b = M.icosphere(2)
    f = np.concatenate([a.faces, b.faces + a.n])
    return M.Mesh("union", a.n + b.n + 5, f.astype(np.int32))   # + 5 isolated vertices


@pytest.mark.parametrize("mesh,cap,seed", [
    (M.grid64(0), 256, 0), (M.grid64(1), 64, 3), (M.shuffle(M.icosphere(4), 2), 100, 2),
    (M.shuffle(M.torus(40, 30, 0.3, 4), 4), 37, 4), (_disconnected_mesh(), 50, 5),
    (M.shuffle(M.grid(20, 20), 6), 1, 6), (M.shuffle(M.grid(15, 15), 7), 10**6, 7)])
def test_patching_invariants(mesh, cap, seed):
    g = _faces_graph(mesh)
    adj = adj_lists(g)
    lab, k = O.patches(g, cap, seed)
    assert lab.min() >= 0 and lab.max() == k - 1
    sizes = np.bincount(lab, minlength=k)
    assert sizes.min() >= 1 and sizes.max() <= cap
    members = [[] for _ in range(k)]
    for v, p in enumerate(lab):
        members[p].append(v)
    for p in range(k):
        assert connected(adj, members[p]), p
    if cap == 1:
        assert k == g.n


# --- contract R11: exact minimum degree --------------------------------------

def test_md_handworked_trace():
    # Degrees 3,3,3,2,2,3. Step 1 takes 3 (degree 2, lower id than 4); step 2
    # takes 1 (degree 2 among {1,2,4}) and adds fill edge 2-5; then 2, 0, 4, 5.
    g = _graph_from_edges(6, [(4, 0), (4, 5), (0, 5), (0, 2), (5, 1), (2, 1), (2, 3), (1, 3)])
    order = O.min_degree(g)
    assert order.tolist() == [3, 1, 2, 0, 4, 5]
    assert fill_of_order(adj_lists(g), order.tolist()) == 1


def test_md_trace_where_fill_decides():
    # C5 labelled 0-3-1-4-2-0, all degrees 2. Step 1 eliminates 0 and adds
    # fill edge 3-2, so 3 and 2 keep degree 2 and the lowest id of degree 2
    # is 1 (without the fill edge 2 and 3 would drop to degree 1 and 2 would
    # come next). Eliminating 1 adds 3-4; the triangle 2, 3, 4 follows.
    g = _graph_from_edges(5, [(0, 3), (3, 1), (1, 4), (4, 2), (2, 0)])
    assert O.min_degree(g).tolist() == [0, 1, 2, 3, 4]


def test_md_special_cases():
    # path and tree: no fill; cycle C_n: n-3 fill edges; clique: no fill.
    n = 9
    path = _graph_from_edges(n, [(i, i + 1) for i in range(n - 1)])
    assert fill_of_order(adj_lists(path), O.min_degree(path).tolist()) == 0
    rng = np.random.default_rng(0)
    for t in range(5):
        edges = [(i, int(rng.integers(0, i))) for i in range(1, 30)]
        tree = _graph_from_edges(30, edges)
        assert fill_of_order(adj_lists(tree), O.min_degree(tree).tolist()) == 0
    for m in range(3, 12):
        cyc = _graph_from_edges(m, [(i, (i + 1) % m) for i in range(m)])
        assert fill_of_order(adj_lists(cyc), O.min_degree(cyc).tolist()) == m - 3
    kn = _graph_from_edges(6, [(i, j) for i in range(6) for j in range(i)])
    assert O.min_degree(kn).tolist() == list(range(6))


@pytest.mark.parametrize("seed", range(8))
def test_md_vs_exhaustive_min_fill(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(5, 9))
    edges = [(i, j) for i in range(n) for j in range(i) if rng.random() < 0.45]
    g = _graph_from_edges(n, edges)
    adj = adj_lists(g)
    md = fill_of_order(adj, O.min_degree(g).tolist())
    best = min_fill_exhaustive(adj)
    assert md >= best
    # minimum degree is optimal when the graph is chordal with a simplicial
    # minimum-degree vertex at each step; at least check it is a valid order
    assert sorted(O.min_degree(g).tolist()) == list(range(n))


# --- symbolic: textbook definitions vs the dense elimination game -------------

def test_symbolic_closed_forms():
    n = 10
    path = _graph_from_edges(n, [(i, i + 1) for i in range(n - 1)])
    s = O.symbolic(path, np.arange(n))
    assert s.parent.tolist() == list(range(1, n)) + [-1]
    assert s.colcount.tolist() == [2] * (n - 1) + [1]
    # star, centre last: no fill; centre first: the leaves become a clique
    star = _graph_from_edges(n, [(0, i) for i in range(1, n)])
    s = O.symbolic(star, np.r_[1:n, 0])
    assert s.parent.tolist() == [n - 1] * (n - 1) + [-1] and s.nnzL == 2 * n - 1
    s = O.symbolic(star, np.arange(n))
    assert s.colcount.tolist() == list(range(n, 0, -1))
    assert s.nnzL == n * (n + 1) // 2 and s.flops == sum(c * c for c in range(1, n + 1))


@pytest.mark.parametrize("seed", range(10))
def test_symbolic_vs_elimination_game(seed):
    rng = np.random.default_rng(seed)
    if seed % 2:
        mesh = M.shuffle(M.torus(7, 6, 0.3, seed), seed)
        g = _faces_graph(mesh)
    else:
        n = int(rng.integers(1, 70))
        edges = [(i, j) for i in range(n) for j in range(i) if rng.random() < 3.0 / max(n, 1)]
        g = _graph_from_edges(n, edges)
    perm = rng.permutation(g.n)
    s = O.symbolic(g, perm)
    L, parent, colcount = elimination_game(adj_lists(g), perm)
    assert np.array_equal(s.parent, parent)
    assert np.array_equal(s.colcount, colcount)
    assert s.nnzL == int(L.sum())
    assert s.flops == int((colcount.astype(np.int64) ** 2).sum())


def test_fp64_cholesky_grid64():
    """P (L_graph + I) P^T on the 64x64 grid: dense FP64 Cholesky has relative
    residual <= 1e-10, and its nonzero count equals the symbolic nnz(L) (an
    M-matrix: no cancellation, so every structural entry is numerically
    nonzero)."""
    mesh = M.grid64(0)
    g = _faces_graph(mesh)
    o = O.order(g, 256, seed=0)
    s = O.symbolic(g, o.perm)
    n = g.n
    A = np.zeros((n, n))
    for v in range(n):
        nb = g.neighbors(v)
        A[v, nb] = -1.0
        A[v, v] = nb.size + 1.0
    B = A[np.ix_(o.perm, o.perm)]
    Lc = np.linalg.cholesky(B)
    res = np.linalg.norm(Lc @ Lc.T - B) / np.linalg.norm(B)
    assert res <= 1e-10
    assert int(np.count_nonzero(Lc)) == s.nnzL
    cc = np.count_nonzero(Lc, axis=0)
    assert np.array_equal(cc, s.colcount)


# --- Sections 2, 4.2, 5: nested-dissection structure invariants ---------------

def _subtree_nodes(t, nn):
    out, st = [], [t]
    while st:
        x = st.pop()
        if x < nn:
            out.append(x); st += [2 * x + 1, 2 * x + 2]
    return out


def _is_ancestor(a, b):
    """tree node a is b or an ancestor of b"""
    while b > a:
        b = (b - 1) // 2
    return a == b


def check_nd_invariants(g, o, default_depth=True):
    n = g.n
    nn = (1 << (o.depth + 1)) - 1
    assert np.array_equal(np.sort(o.perm), np.arange(n))
    assert np.array_equal(o.iperm[o.perm], np.arange(n))
    assert o.node_of.min() >= 0 and o.node_of.max() < nn
    assert np.array_equal(np.bincount(o.node_of, minlength=nn), o.node_size)
    for t in range(nn):
        blk = o.perm[o.node_begin[t]:o.node_begin[t] + o.node_size[t]]
        assert np.all(o.node_of[blk] == t)
    # ND property (Section 2): an edge joins two nodes only if one is an
    # ancestor of the other: no edge between different subtrees.
    src = np.repeat(np.arange(n), np.diff(g.rowptr))
    a, b = o.node_of[src], o.node_of[g.col]
    for x, y in set(zip(a.tolist(), b.tolist())):
        assert _is_ancestor(x, y) or _is_ancestor(y, x), (x, y)
    # separator minimality: each separator vertex has a neighbour of another
    # patch inside one of its node's child subtrees.
    is_leaf = np.array([2 * t + 1 >= nn or o.node_size[2 * t + 1:2 * t + 3].sum() == 0 and
                        all(o.node_size[x] == 0 for x in _subtree_nodes(2 * t + 1, nn) + _subtree_nodes(2 * t + 2, nn))
                        for t in range(nn)])
    for v in range(n):
        t = o.node_of[v]
        if is_leaf[t]:
            continue
        nb = g.neighbors(v)
        ok = [(o.label[u] != o.label[v] and o.node_of[u] != t and _is_ancestor(t, o.node_of[u])) for u in nb]
        assert any(ok), v
    if default_depth:
        # leaves are single patches (patch-level local orderings)
        for t in range(nn):
            if is_leaf[t] and o.node_size[t]:
                blk = o.perm[o.node_begin[t]:o.node_begin[t] + o.node_size[t]]
                assert np.unique(o.label[blk]).size == 1
    return is_leaf


@pytest.mark.parametrize("mesh,cap,seed", [
    (M.grid64(0), 256, 0), (M.grid64(2), 64, 1), (M.shuffle(M.icosphere(4), 3), 128, 3),
    (M.shuffle(M.torus(30, 40, 0.3, 2), 2), 50, 2), (_disconnected_mesh(), 40, 4)])
def test_nd_invariants(mesh, cap, seed):
    g = _faces_graph(mesh)
    o = O.order(g, cap, seed=seed)
    is_leaf = check_nd_invariants(g, o)
    # zero blocks of L between distinct leaves: no etree path leaves a leaf
    # for another leaf's vertex.
    s = O.symbolic(g, o.perm)
    node_pos = o.node_of[o.perm]
    for j in range(0, g.n, 7):
        t = node_pos[j]
        i = s.parent[j]
        while i != -1:
            assert _is_ancestor(node_pos[i], t)
            i = s.parent[i]


@pytest.mark.parametrize("mesh,cap,seed", [
    (M.grid64(0), 64, 0), (M.shuffle(M.icosphere(4), 3), 128, 3), (M.shuffle(M.torus(30, 40, 0.3, 2), 2), 50, 2)])
def test_quotient_weights_match_definition(mesh, cap, seed):
    """Section 5 updates the quotient graph by decrements instead of rebuilding
    it; at every bisected node the weights must equal the definition: the
    number of G-edges between remaining vertices of two different patches,
    the remaining vertices of node t being those of its subtree."""
    g = _faces_graph(mesh)
    o = O.order(g, cap, seed=seed)
    nn = o.node_size.size
    src = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    checked = 0
    for t in range(nn):
        if o.node_qsum[t] < 0:
            continue
        sub = np.zeros(nn, bool)
        sub[_subtree_nodes(t, nn)] = True
        rem = sub[o.node_of]
        m = rem[src] & rem[g.col] & (o.label[src] != o.label[g.col])
        assert int(m.sum()) == o.node_qsum[t], t
        checked += 1
    assert checked > 3


def test_schedule_invariance():
    """Post-order and level-order schedules give the same fill (Section 5)."""
    for mesh, cap in [(M.grid64(0), 256), (M.shuffle(M.icosphere(4), 1), 100)]:
        g = _faces_graph(mesh)
        a = O.order(g, cap, seed=1, schedule=0)
        b = O.order(g, cap, seed=1, schedule=1)
        assert not np.array_equal(a.perm, b.perm)
        assert np.array_equal(a.node_of, b.node_of)
        sa, sb = O.symbolic(g, a.perm), O.symbolic(g, b.perm)
        assert sa.nnzL == sb.nnzL and sa.flops == sb.flops
        check_nd_invariants(g, b)


def test_cap_one_is_classical_nd():
    """Every patch a single vertex: the method is nested dissection on G itself
    (Section 4 overview)."""
    g = _faces_graph(M.shuffle(M.grid(12, 11), 3))
    o = O.order(g, 1, seed=3)
    assert o.k == g.n
    check_nd_invariants(g, o)


def test_single_patch_is_minimum_degree():
    """One patch: depth 0, the root leaf holds every vertex, perm = MD of G."""
    mesh = M.shuffle(M.grid(9, 8), 4)
    g = _faces_graph(mesh)
    for seed in range(200):
        o = O.order(g, 10**6, seed=seed)
        if o.k == 1:
            break
    assert o.k == 1 and o.depth == 0
    assert np.array_equal(o.perm, O.min_degree(g))


def test_nd_level_limits_depth():
    g = _faces_graph(M.grid64(0))
    o = O.order(g, 64, seed=0, nd_level=3)
    assert o.depth == 3 and o.node_size.size == 15
    check_nd_invariants(g, o, default_depth=False)


def test_dof_expansion_matches_direct_symbolic():
    """Section 6.5: the ordering of the compressed graph expanded to b DOFs
    gives exactly the symbolic structure of the DOF matrix."""
    g = _faces_graph(M.shuffle(M.torus(8, 7, 0.3, 5), 5))
    n, b = g.n, 3
    o = O.order(g, 20, seed=5)
    s = O.symbolic(g, o.perm)
    rows = []
    for i in range(n * b):
        v = i // b
        nb = [b * u + c for u in g.neighbors(v).tolist() for c in range(b)]
        nb += [b * v + c for c in range(b) if b * v + c != i]
        rows.append(sorted(nb))
    dg = O.Graph(np.cumsum([0] + [len(r) for r in rows]).astype(np.int32), np.array(sum(rows, []), np.int32))
    pd, ad, cd = O.dof_expand(b, o.perm, s.parent, s.colcount)
    sd = O.symbolic(dg, pd)
    assert np.array_equal(sd.parent, ad) and np.array_equal(sd.colcount, cd)
    assert sd.nnzL == b * b * s.nnzL - n * b * (b - 1) // 2


def test_empty_and_tiny_inputs():
    g = O.graph_from_faces(np.zeros((0, 3), np.int32), 0)
    o = O.order(g, 16)
    assert o.perm.size == 0
    g = O.graph_from_faces(np.zeros((0, 3), np.int32), 7)     # isolated vertices
    o = O.order(g, 16, seed=1)
    assert o.k == 7
    check_nd_invariants(g, o)
    s = O.symbolic(g, o.perm)
    assert s.nnzL == 7 and np.all(s.parent == -1)


def test_supplied_patches():
    """Algorithm 1 with the patch partition supplied (Section 4, opening):
    given the patches the method computes itself it reproduces them exactly;
    one group is plain minimum degree of G; disconnected groups and empty
    labels (zero-weight patches, which take no part) still give a valid
    dissection."""
    mesh = M.shuffle(M.torus(30, 22, 0.3, 9), 9)
    g = _faces_graph(mesh)
    o = O.order(g, 60, seed=9)
    same = O.order_given(g, o.label, o.k)
    for f in ("label", "node_of", "perm", "iperm", "node_begin", "node_size"):
        assert np.array_equal(getattr(o, f), getattr(same, f)), f
    one = O.order_given(g, np.zeros(g.n, np.int32), 1)
    assert one.depth == 0 and np.array_equal(one.perm, O.min_degree(g))
    lab = (np.arange(g.n) * 7919 % 13).astype(np.int32)        # 13 scattered, disconnected groups
    lab[lab == 5] = 3                                           # label 5 left empty
    d = O.order_given(g, lab, 13)
    assert d.k == 13 and np.array_equal(d.label, lab)
    assert np.array_equal(np.sort(d.perm), np.arange(g.n))
    check_nd_invariants(g, d)
    with pytest.raises(ValueError):
        O.order_given(g, np.full(g.n, 13, np.int32), 13)
