"""Pins of the learned-priority oracle (oracle/gnn.py) against definitions,
hand-computed values, brute force and the fill-monotonicity theorem."""
from fractions import Fraction

import numpy as np
import pytest

import meshgen
import oracle as O
from oracle import gnn as G
from tests import brute


def _grid(seed=0):
    m = meshgen.grid64(seed)
    g = O.graph_from_faces(m.faces, m.n)
    return g, O.order(g, 256, seed=seed)


def test_rne_div_matches_exact_rounding():
    rng = np.random.default_rng(1)
    a = rng.integers(0, 10**6, 2000)
    b = rng.integers(1, 300, 2000)
    got = G.rne_div(a, b)
    # Python's round() of an exact fraction rounds half to even
    want = np.array([round(Fraction(int(x), int(y))) for x, y in zip(a, b)])
    assert (got == want).all()
    assert G.rne_div(5, 2) == 2 and G.rne_div(7, 2) == 4 and G.rne_div(320, 128) == 2


def test_leaves_definition():
    # sizes by node (binary tree in an array): node 1 has non-empty children
    o = O.Ordering(1, 2, np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(7, np.int32),
                   np.array([5, 3, 0, 2, 1, 0, 0], np.int32), np.zeros(7))
    assert G.leaves(o) == [3, 4]
    # a node whose descendants are all empty is a leaf; empty nodes are not
    o.node_size = np.array([4, 2, 0, 0, 0, 0, 0], np.int32)
    assert G.leaves(o) == [1]


def _manual(adj_edges, n, node_of_pos, sizes):
    """Graph + hand-made ordering with perm = identity."""
    rows = [[] for _ in range(n)]
    for a, b in adj_edges:
        rows[a].append(b)
        rows[b].append(a)
    rp = np.zeros(n + 1, np.int32)
    for v in range(n):
        rp[v + 1] = rp[v] + len(rows[v])
    col = np.array([u for r in rows for u in sorted(r)], np.int32)
    g = O.Graph(rp, col)
    begin = np.zeros(len(sizes), np.int32)
    for t in range(len(sizes)):
        begin[t] = [p for p in range(n) if node_of_pos[p] == t][0] if sizes[t] else 0
    perm = np.arange(n, dtype=np.int32)
    return g, O.Ordering(1, 1, np.zeros(n, np.int32), np.array(node_of_pos, np.int32), perm, perm.copy(),
                         begin, np.array(sizes, np.int32), np.zeros(len(sizes)))


def test_features_hand_computed():
    # path 0-1-2-3-4-5; node 0 (separator) = {3}; leaf 1 = {0,1,2}; leaf 2 = {4,5}
    g, o = _manual([(0, 1), (1, 2), (2, 3), (3, 4), (4, 5)], 6, [1, 1, 1, 0, 2, 2], [1, 3, 2])
    X = G.features(g, o, cap=8)
    # leaf {0,1,2}: boundary = {2} (neighbour 3 outside); depths 2,1,0; dmax = 2
    assert X[0].tolist() == [8, 8, 0, 43, 24, 64]     # 64*2/3 = 42.67 -> 43; 64*3/8 = 24
    assert X[1].tolist() == [16, 16, 0, 21, 24, 64]   # 64/3 = 21.3 -> 21
    assert X[2].tolist() == [8, 16, 64, 0, 24, 64]
    # leaf {4,5}: boundary {4}; depths 0,1; dmax = 1; size 2/8 -> 16
    assert X[4].tolist() == [8, 16, 64, 0, 16, 64]
    assert X[5].tolist() == [8, 8, 0, 32, 16, 64]
    assert X[3].tolist() == [0] * 6                    # separator: no features


def _two_vertex_leaf():
    g, o = _manual([(0, 1), (1, 2)], 3, [1, 1, 0], [1, 2, 0])
    lg = G.leaf_graph(g, o)
    X = np.zeros((3, 6), np.int64)
    X[0] = [64, 0, 0, 0, 0, 64]
    X[1] = [128, 0, 0, 0, 0, 64]
    return g, o, lg, X


def test_forward_q_hand_computed_ties_to_even():
    g, o, lg, X = _two_vertex_leaf()
    z = lambda *s: np.zeros(s, np.int64)
    qp = G.QParams(z(32, 6), z(32, 6), z(32), z(32, 32), z(32, 32), z(32), z(32), 5)
    qp.w1s[0, 0], qp.w1n[0, 0] = 2, 1        # unit 0: 2/128 x + 1/128 mean(x)
    qp.w1s[1, 0] = -1                         # unit 1: negative -> ReLU zero
    qp.w2s[0, 0] = 128                        # passes unit 0 through
    qp.w3[0] = 3
    S = G.forward_q(qp, X, lg)
    # vertex 0: Z = 2*64 + 1*128 = 256 -> 256/128 = 2 ; vertex 1: 2*128 + 64 = 320 -> 2.5 -> 2 (even)
    # layer 2: Z = 128*2 = 256 -> 2 ; S = 3*2 + 5 = 11 for both (half-up would give 14 for vertex 1)
    assert S[0] == 11 and S[1] == 11 and S[2] == 0


def test_forward_q_constant_without_weights_and_local_without_messages():
    g, o = _grid()
    lg = G.leaf_graph(g, o)
    X = G.features(g, o, 256, lg)
    d = meshgen.gnn_weights(3)
    zero = {k: np.zeros_like(np.asarray(v)) for k, v in d.items()}
    zero["c"] = np.array(77)
    S = G.forward_q(G.QParams.from_dict(zero), X, lg)
    assert (S[lg.is_leaf] == 77).all()
    # no neighbour weights: a vertex's score depends on its own features only
    loc = dict(d)
    loc["w1n"] = np.zeros_like(d["w1n"])
    loc["w2n"] = np.zeros_like(d["w2n"])
    qp = G.QParams.from_dict(loc)
    S1 = G.forward_q(qp, X, lg)
    p = int(np.nonzero(lg.is_leaf)[0][10])
    nbrs = lg.col[lg.rowptr[p]:lg.rowptr[p + 1]]
    X2 = X.copy()
    X2[nbrs] = (X2[nbrs] + 17) % 256
    S2 = G.forward_q(qp, X2, lg)
    assert S2[p] == S1[p]
    assert any(S2[q] != S1[q] for q in nbrs)


def test_forward_q_equivariant_and_exact_range():
    g, o = _grid(1)
    lg = G.leaf_graph(g, o)
    X = G.features(g, o, 256, lg)
    qp = G.QParams.from_dict(meshgen.gnn_weights(5))
    qp.check()
    S = G.forward_q(qp, X, lg)
    # relabel the vertices: same ordering up to the relabelling -> same scores per vertex
    rng = np.random.default_rng(0)
    pi = rng.permutation(g.n).astype(np.int32)
    m = meshgen.grid64(1)
    g2 = O.graph_from_faces(pi[m.faces], m.n)
    o2 = O.order(g2, 256, seed=1)
    lg2 = G.leaf_graph(g2, o2)
    S2 = G.forward_q(qp, G.features(g2, o2, 256, lg2), lg2)
    # compare per original vertex when the two trees hold the same vertex sets
    by_v1 = {int(o.perm[p]): int(S[p]) for p in range(g.n) if lg.is_leaf[p]}
    inv = np.empty_like(pi)
    inv[pi] = np.arange(g.n)
    by_v2 = {int(inv[o2.perm[p]]): int(S2[p]) for p in range(g.n) if lg2.is_leaf[p]}
    common = set(by_v1) & set(by_v2)
    assert len(common) > 0
    # every dot product stays far inside FP32's exact-integer range
    bound = 64 * G.W_MAX * G.H_MAX + G.B_MAX
    assert bound < 2 ** 24


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_keyed_min_degree_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    m = meshgen.grid(5, 4)
    g = O.graph_from_faces(m.faces, m.n)
    adj = brute.adj_lists(g)
    verts = sorted(rng.choice(m.n, 14, replace=False).tolist())
    key = rng.integers(0, 4, len(verts)).astype(np.uint32)   # many ties
    got = O.min_degree_keyed(g, verts, key)
    assert got.tolist() == brute.md_keyed_brute(adj, verts, key.tolist())
    # equal keys reduce to plain minimum degree (ties to the smaller id)
    plain = O.min_degree_keyed(g, verts, np.zeros(len(verts), np.uint32))
    assert plain.tolist() == brute.md_keyed_brute(adj, verts, [0] * len(verts))


def test_leaf_fill_shortcut_equals_elimination_game():
    g, o = _grid(2)
    adj = brute.adj_lists(g)
    lv = G.leaves(o)
    key = np.array([O.tie_key(3, v) for v in range(g.n)], np.uint32)
    perm = G.keyed_perm(g, o, lv, key)
    fills = G.leaf_fills(g, o, perm, lv)
    for i, t in enumerate(lv[:12]):
        b, m = int(o.node_begin[t]), int(o.node_size[t])
        assert fills[i] == brute.leaf_fill_brute(adj, perm[b:b + m].tolist())


@pytest.mark.parametrize("seed", [0, 1, 4])
def test_learned_never_worse_than_plain(seed):
    g, o = _grid(seed)
    qp = G.QParams.from_dict(meshgen.gnn_weights(10 + seed))
    L = G.order_learned(g, o, qp, 256)
    plain = O.symbolic(g, o.perm)
    learned = O.symbolic(g, L.perm)
    assert learned.nnzL <= plain.nnzL
    assert learned.nnzL == plain.nnzL - int((L.fill_plain - L.fill_learned)[L.kept].sum())
    assert sorted(L.perm.tolist()) == list(range(g.n))
    # separator columns do not move and keep their counts
    sep = np.ones(g.n, bool)
    for t in L.leaves:
        sep[o.node_begin[t]:o.node_begin[t] + o.node_size[t]] = False
    assert (learned.colcount[sep] == plain.colcount[sep]).all()


def test_learned_with_constant_scores_is_plain():
    g, o = _grid(3)
    d = {k: np.zeros_like(np.asarray(v)) for k, v in meshgen.gnn_weights(0).items()}
    L = G.order_learned(g, o, G.QParams.from_dict(d), 256)
    assert (L.perm == o.perm).all() and not L.kept.any()


def test_targets_pick_the_lowest_fill():
    g, o = _grid(0)
    T = G.targets(g, o, n_seeds=8)
    assert T.fills.shape[0] == 9
    assert (T.fills[T.best_r, np.arange(T.fills.shape[1])] == T.fills.min(axis=0)).all()
    lv = G.leaves(o)
    plain = G.leaf_fills(g, o, o.perm, lv)
    assert (T.fills[0] == plain).all()
    for t in lv:
        b, m = int(o.node_begin[t]), int(o.node_size[t])
        assert sorted(T.rank[b:b + m].tolist()) == list(range(m))
    assert (T.target[T.rank >= 0] <= 1.0).all() and (T.target >= 0).all()


def _tiny_float_problem(seed):
    g, o = _grid(seed)
    lg = G.leaf_graph(g, o)
    X = G.features(g, o, 256, lg) / 64.0
    T = G.targets(g, o, 2).target
    P = {k: np.asarray(v, np.float64) for k, v in meshgen.gnn_weights(seed, quantized=False).items()}
    return P, X, lg, T


def test_gradient_matches_finite_differences():
    P, X, lg, T = _tiny_float_problem(0)
    loss, g = G.loss_and_grad(P, X, lg, T)
    rng = np.random.default_rng(0)
    eps = 1e-6
    for k in P:
        flat = P[k].reshape(-1)
        for idx in rng.choice(flat.size, min(4, flat.size), replace=False):
            Pp = {kk: vv.copy() for kk, vv in P.items()}
            Pm = {kk: vv.copy() for kk, vv in P.items()}
            Pp[k].reshape(-1)[idx] += eps
            Pm[k].reshape(-1)[idx] -= eps
            fd = (G.loss_and_grad(Pp, X, lg, T)[0] - G.loss_and_grad(Pm, X, lg, T)[0]) / (2 * eps)
            an = np.asarray(g[k]).reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 + 1e-4 * abs(fd), (k, idx, fd, an)


def test_sgd_decreases_the_loss():
    P, X, lg, T = _tiny_float_problem(1)
    l0, g = G.loss_and_grad(P, X, lg, T)
    for _ in range(5):
        P = G.sgd_step(P, g, 0.02)
        l1, g = G.loss_and_grad(P, X, lg, T)
    assert l1 < l0


def test_quantise_rounds_to_the_grid():
    d = meshgen.gnn_weights(2, quantized=False)
    q = G.quantise(d)
    assert (q.w1s == np.clip(np.rint(d["w1s"] * 128), -255, 255)).all()
    assert q.c == int(np.rint(d["c"] * 8192))


def test_tie_key_is_high_half_of_seed_hash():
    for r, v in [(1, 0), (3, 17), (8, 123456)]:
        assert O.tie_key(r, v) == O.seed_hash(r, v) >> 32
