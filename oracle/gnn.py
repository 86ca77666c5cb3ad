"""Oracle of the learned elimination priorities (the learned part of the
ordering). TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
benchmark's CPU legs use this module; the library never does.

The paper orders each patch by (approximate) minimum degree and says nothing
about learned orderings; this part adds, per leaf of the nested-dissection
tree, a second candidate order whose minimum-degree ties are broken by a small
message-passing network's scores, and keeps whichever of the two has the
smaller exact fill. Each reading below is stated where it is implemented:

  L1 leaves: tree nodes with vertices and no non-empty descendant (with the
     default tree depth, the single-patch leaves of Section 4.2) and at most
     512 vertices (a larger leaf, possible only with patch caps above 512,
     keeps its plain order).
  L2 features of a leaf vertex v on the leaf's induced subgraph H (integer
     codes q, value q/64, q clamped to [0, 255]):
       deg_H(v)/8, deg_G(v)/8, [v has a neighbour outside the leaf],
       depth(v)/(dmax+1) (hop distance in H to the nearest boundary vertex;
       dmax+1 for vertices with no boundary vertex in their component),
       |leaf|/cap, 1.
  L3 network: two layers h' = ReLU(Ws h + Wn mean_{u in N_H(v)} h_u + b) of
     width 32 and a scalar head s = w.h + c, computed on a fixed-point grid
     that BF16 represents exactly: activations q/64 (q in [0, 255]), weights
     q/128 (|q| <= 255), biases and scores q/8192. Every dot product is then
     an exact integer in units of 1/8192 (far below 2^24), so FP32
     accumulation on any hardware gives the same bits. The neighbour mean and
     the re-quantisation of each layer round to nearest, ties to even, in
     integer arithmetic.
  L4 learned order: exact minimum degree on H with ties to the smaller
     (key, id), key = 2^23 - S (the highest score goes first).
  L5 fill of a leaf order: the sum of the column counts of the leaf's
     columns, i.e. the elimination game on the leaf plus its neighbouring
     separator vertices. A leaf's column counts depend on its own order only
     (separator counts depend on the vertex sets below them, not on their
     order), so the fills of all leaves come from one symbolic factorisation
     of a permutation that uses the candidate order in every leaf.
  L6 choice: the learned order is kept iff its fill is smaller; ties keep
     plain minimum degree. Hence nnz(L) never exceeds the plain method's.
  L7 training targets: candidates are plain MD (r = 0) and MD with seeded
     tie-break keys r = 1..8 (the high 32 bits of SplitMix64 at r*gamma + v);
     the lowest fill wins (ties to the lower r); the target of a vertex at
     rank k of the winning order of an m-vertex leaf is (m-1-k)/(m-1)
     (1 for m = 1).
  L8 training: the same network in float without the grid (activations
     clamped to [0, 255/64] like the codes), loss = mean squared error over
     leaf vertices, plain gradient descent, weights quantised to the grid
     afterwards by rounding to nearest.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import Graph, Ordering, local_orders_keyed, symbolic, tie_key

F_IN = 6
HID = 32
Q_X = 64            # activation grid: value = q / 64
Q_W = 128           # weight grid: value = q / 128
Q_B = Q_X * Q_W     # bias / score grid: value = q / 8192
H_MAX = 255         # largest activation code
W_MAX = 255         # largest weight code magnitude
B_MAX = 1 << 20     # largest bias code magnitude
KEY_BIAS = 1 << 23  # learned key = KEY_BIAS - S
LEAF_MAX = 512      # largest leaf that gets a learned candidate


def rne_div(a, b):
    """a / b rounded to nearest, ties to even, for integers a >= 0, b > 0
    (numpy arrays or ints)."""
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    q, r = np.divmod(a, b)
    up = (2 * r > b) | ((2 * r == b) & (q % 2 == 1))
    return q + up.astype(np.int64)


# ---------------------------------------------------------------------------
# L1 leaves and their induced subgraphs
# ---------------------------------------------------------------------------

def leaves(o: Ordering) -> list[int]:
    """Nodes with vertices and no non-empty descendant (L1)."""
    nn = o.node_size.size
    sub = o.node_size.astype(np.int64).copy()
    for t in range(nn - 1, -1, -1):
        for c in (2 * t + 1, 2 * t + 2):
            if c < nn:
                sub[t] += sub[c]
    return [t for t in range(nn) if 0 < o.node_size[t] <= LEAF_MAX and sub[t] == o.node_size[t]]


@dataclass
class LeafGraph:
    """Leaf vertices indexed by their plain position p in perm; arrays of
    length n (rows of non-leaf positions stay empty)."""
    n: int
    is_leaf: np.ndarray        # bool [n] per position
    leaf_of: np.ndarray        # node id per position (-1 off leaves)
    rowptr: np.ndarray         # CSR over positions of the within-leaf neighbours
    col: np.ndarray            # neighbour positions
    deg_g: np.ndarray          # degree in G per position
    boundary: np.ndarray       # bool: a neighbour outside the leaf
    leaf_list: list = field(default_factory=list)


def leaf_graph(g: Graph, o: Ordering) -> LeafGraph:
    n = g.n
    is_leaf = np.zeros(n, bool)
    leaf_of = np.full(n, -1, np.int64)
    lv = leaves(o)
    for t in lv:
        b, m = int(o.node_begin[t]), int(o.node_size[t])
        is_leaf[b:b + m] = True
        leaf_of[b:b + m] = t
    rows = [[] for _ in range(n)]
    deg_g = np.zeros(n, np.int64)
    boundary = np.zeros(n, bool)
    for p in range(n):
        if not is_leaf[p]:
            continue
        v = int(o.perm[p])
        nb = g.neighbors(v)
        deg_g[p] = nb.size
        for u in nb:
            q = int(o.iperm[u])
            if leaf_of[q] == leaf_of[p]:
                rows[p].append(q)
            else:
                boundary[p] = True
    rp = np.zeros(n + 1, np.int64)
    for p in range(n):
        rp[p + 1] = rp[p] + len(rows[p])
    col = np.array([q for r in rows for q in r], np.int64)
    return LeafGraph(n, is_leaf, leaf_of, rp, col, deg_g, boundary, lv)


# ---------------------------------------------------------------------------
# L2 features
# ---------------------------------------------------------------------------

def features(g: Graph, o: Ordering, cap: int, lg: LeafGraph | None = None) -> np.ndarray:
    """Integer feature codes [n, 6] per position (zero rows off leaves)."""
    lg = lg or leaf_graph(g, o)
    n = g.n
    X = np.zeros((n, F_IN), np.int64)
    for t in lg.leaf_list:
        b, m = int(o.node_begin[t]), int(o.node_size[t])
        ps = list(range(b, b + m))
        # hop distance to the nearest boundary vertex inside the leaf (BFS)
        depth = {p: None for p in ps}
        frontier = [p for p in ps if lg.boundary[p]]
        for p in frontier:
            depth[p] = 0
        d = 0
        while frontier:
            nxt = []
            for p in frontier:
                for q in lg.col[lg.rowptr[p]:lg.rowptr[p + 1]]:
                    q = int(q)
                    if depth[q] is None:
                        depth[q] = d + 1
                        nxt.append(q)
            frontier = nxt
            d += 1
        finite = [x for x in depth.values() if x is not None]
        dmax = max(finite) if finite else 0
        for p in ps:
            dh = int(lg.rowptr[p + 1] - lg.rowptr[p])
            dp = depth[p] if depth[p] is not None else dmax + 1
            X[p, 0] = min(8 * dh, H_MAX)
            X[p, 1] = min(8 * int(lg.deg_g[p]), H_MAX)
            X[p, 2] = Q_X if lg.boundary[p] else 0
            X[p, 3] = min(int(rne_div(Q_X * dp, dmax + 1)), H_MAX)
            X[p, 4] = min(int(rne_div(Q_X * m, cap)), H_MAX)
            X[p, 5] = Q_X
    return X


# ---------------------------------------------------------------------------
# L3 quantised network
# ---------------------------------------------------------------------------

@dataclass
class QParams:
    w1s: np.ndarray  # [32, 6] codes, value q/128
    w1n: np.ndarray  # [32, 6]
    b1: np.ndarray   # [32] codes, value q/8192
    w2s: np.ndarray  # [32, 32]
    w2n: np.ndarray  # [32, 32]
    b2: np.ndarray   # [32]
    w3: np.ndarray   # [32]
    c: int           # value c/8192

    @staticmethod
    def from_dict(d: dict) -> "QParams":
        a = {k: np.asarray(v, np.int64) for k, v in d.items()}
        return QParams(a["w1s"], a["w1n"], a["b1"], a["w2s"], a["w2n"], a["b2"], a["w3"], int(a["c"]))

    def check(self):
        for k in ("w1s", "w1n", "w2s", "w2n", "w3"):
            assert np.abs(getattr(self, k)).max(initial=0) <= W_MAX, k
        for k in ("b1", "b2"):
            assert np.abs(getattr(self, k)).max(initial=0) <= B_MAX, k
        assert abs(self.c) <= B_MAX


def neighbour_mean_q(H: np.ndarray, lg: LeafGraph) -> np.ndarray:
    """Mean of the neighbours' codes, rounded to nearest even (0 without
    neighbours)."""
    M = np.zeros_like(H)
    for p in range(lg.n):
        r0, r1 = lg.rowptr[p], lg.rowptr[p + 1]
        if r1 > r0:
            M[p] = rne_div(H[lg.col[r0:r1]].sum(axis=0), r1 - r0)
    return M


def requantise(Z: np.ndarray) -> np.ndarray:
    """ReLU, then units of 1/8192 -> activation codes (1/64), clamped."""
    return np.minimum(rne_div(np.maximum(Z, 0), Q_W), H_MAX)


def forward_q(qp: QParams, X: np.ndarray, lg: LeafGraph) -> np.ndarray:
    """Scores S (integer, value S/8192) per position; exact integer math."""
    M0 = neighbour_mean_q(X, lg)
    Z1 = X @ qp.w1s.T + M0 @ qp.w1n.T + qp.b1
    H1 = requantise(Z1)
    M1 = neighbour_mean_q(H1, lg)
    Z2 = H1 @ qp.w2s.T + M1 @ qp.w2n.T + qp.b2
    H2 = requantise(Z2)
    S = H2 @ qp.w3 + qp.c
    return np.where(lg.is_leaf, S, 0)


def quantise(params: dict) -> QParams:
    """Float weights -> codes by rounding to nearest (L8)."""
    def q(x, scale, lim):
        return np.clip(np.rint(np.asarray(x, np.float64) * scale), -lim, lim).astype(np.int64)
    return QParams(q(params["w1s"], Q_W, W_MAX), q(params["w1n"], Q_W, W_MAX), q(params["b1"], Q_B, B_MAX),
                   q(params["w2s"], Q_W, W_MAX), q(params["w2n"], Q_W, W_MAX), q(params["b2"], Q_B, B_MAX),
                   q(params["w3"], Q_W, W_MAX), int(q(params["c"], Q_B, B_MAX)))


# ---------------------------------------------------------------------------
# L4-L6 learned leaf orders and the exact-fill choice
# ---------------------------------------------------------------------------

def leaf_fills(g: Graph, o: Ordering, perm: np.ndarray, lv: list[int]) -> np.ndarray:
    """Per leaf (in lv order): the sum of its columns' counts under perm (L5)."""
    sym = symbolic(g, perm)
    return np.array([int(sym.colcount[o.node_begin[t]:o.node_begin[t] + o.node_size[t]].sum()) for t in lv],
                    np.int64)


def keyed_perm(g: Graph, o: Ordering, lv: list[int], key_of_vertex) -> np.ndarray:
    """The plain perm with every leaf reordered by keyed minimum degree."""
    ptr = [0]
    verts = []
    for t in lv:
        b, m = int(o.node_begin[t]), int(o.node_size[t])
        verts.extend(int(v) for v in o.perm[b:b + m])
        ptr.append(len(verts))
    orders = local_orders_keyed(g, np.array(ptr), np.array(verts, np.int64), key_of_vertex)
    perm = o.perm.copy()
    for i, t in enumerate(lv):
        b = int(o.node_begin[t])
        perm[b:b + int(o.node_size[t])] = orders[ptr[i]:ptr[i + 1]]
    return perm


@dataclass
class Learned:
    perm: np.ndarray
    iperm: np.ndarray
    leaves: list
    kept: np.ndarray          # bool per leaf: learned order kept
    fill_plain: np.ndarray    # per leaf
    fill_learned: np.ndarray  # per leaf
    scores: np.ndarray        # S per position (plain positions)


def order_learned(g: Graph, o: Ordering, qp: QParams, cap: int) -> Learned:
    """L1-L6 on top of the plain ordering o."""
    lg = leaf_graph(g, o)
    X = features(g, o, cap, lg)
    S = forward_q(qp, X, lg)
    key = np.zeros(g.n, np.uint32)
    for p in range(g.n):
        if lg.is_leaf[p]:
            key[o.perm[p]] = np.uint32(KEY_BIAS - int(S[p]))
    lv = lg.leaf_list
    perm_l = keyed_perm(g, o, lv, key)
    fp = leaf_fills(g, o, o.perm, lv)
    fl = leaf_fills(g, o, perm_l, lv)
    kept = fl < fp
    perm = o.perm.copy()
    for i, t in enumerate(lv):
        if kept[i]:
            b, m = int(o.node_begin[t]), int(o.node_size[t])
            perm[b:b + m] = perm_l[b:b + m]
    iperm = np.empty_like(perm)
    iperm[perm] = np.arange(g.n, dtype=perm.dtype)
    return Learned(perm, iperm, lv, kept, fp, fl, S)


# ---------------------------------------------------------------------------
# L7 training targets
# ---------------------------------------------------------------------------

@dataclass
class Targets:
    rank: np.ndarray     # rank of each position's vertex in its leaf's best order (-1 off leaves)
    target: np.ndarray   # float64 target per position (0 off leaves)
    best_r: np.ndarray   # winning candidate per leaf
    fills: np.ndarray    # [n_cand, n_leaves]


def targets(g: Graph, o: Ordering, n_seeds: int = 8) -> Targets:
    lg = leaf_graph(g, o)
    lv = lg.leaf_list
    perms, fills = [], []
    for r in range(n_seeds + 1):
        key = None if r == 0 else np.array([tie_key(r, v) for v in range(g.n)], np.uint32)
        pr = keyed_perm(g, o, lv, key)
        perms.append(pr)
        fills.append(leaf_fills(g, o, pr, lv))
    fills = np.array(fills)
    best = np.argmin(fills, axis=0)           # first minimum: ties to the lower r
    rank = np.full(g.n, -1, np.int64)
    tgt = np.zeros(g.n)
    for i, t in enumerate(lv):
        b, m = int(o.node_begin[t]), int(o.node_size[t])
        order = perms[best[i]][b:b + m]
        pos_of = {int(v): k for k, v in enumerate(order)}
        for p in range(b, b + m):
            k = pos_of[int(o.perm[p])]
            rank[p] = k
            tgt[p] = 1.0 if m == 1 else (m - 1 - k) / (m - 1)
    return Targets(rank, tgt, best, fills)


# ---------------------------------------------------------------------------
# L8 float network, loss, gradients, SGD
# ---------------------------------------------------------------------------

HF_MAX = H_MAX / Q_X   # float activation clamp


def _mean(H, lg):
    M = np.zeros_like(H)
    for p in range(lg.n):
        r0, r1 = lg.rowptr[p], lg.rowptr[p + 1]
        if r1 > r0:
            M[p] = H[lg.col[r0:r1]].mean(axis=0)
    return M


def _mean_t(G, lg):
    """Adjoint of _mean: out[u] = sum over v with u in N(v) of G[v] / deg(v)."""
    out = np.zeros_like(G)
    for p in range(lg.n):
        r0, r1 = lg.rowptr[p], lg.rowptr[p + 1]
        for q in lg.col[r0:r1]:
            out[q] += G[p] / (r1 - r0)
    return out


def float_forward(P: dict, X: np.ndarray, lg: LeafGraph) -> dict:
    """X: float features [n, 6] (codes / 64)."""
    M0 = _mean(X, lg)
    Z1 = X @ P["w1s"].T + M0 @ P["w1n"].T + P["b1"]
    H1 = np.clip(Z1, 0.0, HF_MAX)
    M1 = _mean(H1, lg)
    Z2 = H1 @ P["w2s"].T + M1 @ P["w2n"].T + P["b2"]
    H2 = np.clip(Z2, 0.0, HF_MAX)
    s = H2 @ P["w3"] + P["c"]
    return dict(X=X, M0=M0, Z1=Z1, H1=H1, M1=M1, Z2=Z2, H2=H2, s=s)


def loss_and_grad(P: dict, X: np.ndarray, lg: LeafGraph, T: np.ndarray) -> tuple[float, dict]:
    """Mean squared error over leaf positions and its exact gradient."""
    f = float_forward(P, X, lg)
    mask = lg.is_leaf.astype(np.float64)
    N = max(mask.sum(), 1.0)
    r = (f["s"] - T) * mask
    loss = float((r * r).sum() / N)
    ds = 2.0 * r / N
    g = {}
    g["w3"] = f["H2"].T @ ds
    g["c"] = np.array(ds.sum())
    dZ2 = np.outer(ds, P["w3"]) * ((f["Z2"] > 0) & (f["Z2"] < HF_MAX))
    g["w2s"] = dZ2.T @ f["H1"]
    g["w2n"] = dZ2.T @ f["M1"]
    g["b2"] = dZ2.sum(axis=0)
    dH1 = dZ2 @ P["w2s"] + _mean_t(dZ2 @ P["w2n"], lg)
    dZ1 = dH1 * ((f["Z1"] > 0) & (f["Z1"] < HF_MAX))
    g["w1s"] = dZ1.T @ f["X"]
    g["w1n"] = dZ1.T @ f["M0"]
    g["b1"] = dZ1.sum(axis=0)
    return loss, g


def sgd_step(P: dict, g: dict, lr: float) -> dict:
    return {k: P[k] - lr * g[k] for k in P}
