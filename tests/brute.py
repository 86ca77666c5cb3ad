"""Brute-force and textbook checks used to pin the oracle (tiny inputs only).

Nothing here is a restatement of the oracle's code path: each function computes
its quantity straight from a definition (one BFS per source, the dense
elimination game, exhaustive search over orderings)."""
from __future__ import annotations

import itertools
from collections import deque

import numpy as np


def adj_lists(g) -> list[list[int]]:
    return [g.col[g.rowptr[v]:g.rowptr[v + 1]].tolist() for v in range(g.n)]


def bfs_from(adj, s, group=None):
    """Hop distances from s (-1 = unreached), edges restricted to equal group."""
    d = [-1] * len(adj)
    d[s] = 0
    q = deque([s])
    while q:
        u = q.popleft()
        for v in adj[u]:
            if group is not None and group[u] != group[v]:
                continue
            if d[v] < 0:
                d[v] = d[u] + 1
                q.append(v)
    return d


def voronoi_brute(adj, src, rank, group=None):
    """dist(v) = min over sources of BFS distance; label = min rank at that
    distance; each source BFS'd on its own."""
    n = len(adj)
    best = [(10**9, -1)] * n
    for s, r in zip(src, rank):
        d = bfs_from(adj, s, group)
        for v in range(n):
            if d[v] >= 0 and (d[v], r) < best[v]:
                best[v] = (d[v], r)
    dist = np.array([b[0] if b[1] >= 0 else -1 for b in best])
    lab = np.array([b[1] for b in best])
    return dist, lab


def connected(adj, verts) -> bool:
    vs = set(verts)
    if not vs:
        return True
    s = next(iter(vs))
    seen = {s}
    q = [s]
    while q:
        u = q.pop()
        for v in adj[u]:
            if v in vs and v not in seen:
                seen.add(v)
                q.append(v)
    return len(seen) == len(vs)


def elimination_game(adj, perm):
    """Dense elimination of P (G + I) P^T in order: returns the filled lower
    pattern as a boolean matrix in new indices, then parent and colcount read
    directly from it (parent[j] = first row below j, colcount[j] = nonzeros
    of column j including the diagonal)."""
    n = len(adj)
    iperm = np.empty(n, np.int64)
    iperm[np.asarray(perm)] = np.arange(n)
    M = np.zeros((n, n), bool)
    for u in range(n):
        for v in adj[u]:
            M[iperm[u], iperm[v]] = True
    np.fill_diagonal(M, True)
    for j in range(n):
        rows = np.nonzero(M[j + 1:, j])[0] + j + 1
        if rows.size:
            M[np.ix_(rows, rows)] = True
    L = np.tril(M)
    parent = np.full(n, -1)
    colcount = L.sum(0).astype(np.int64)
    for j in range(n):
        r = np.nonzero(L[j + 1:, j])[0]
        if r.size:
            parent[j] = j + 1 + r[0]
    return L, parent, colcount


def fill_of_order(adj, order) -> int:
    """Number of fill edges created by eliminating in `order` (bitmask game)."""
    n = len(adj)
    nb = [0] * n
    for u in range(n):
        for v in adj[u]:
            nb[u] |= 1 << v
    alive = (1 << n) - 1
    fill = 0
    for p in order:
        ns = nb[p] & alive & ~(1 << p)
        members = [i for i in range(n) if ns >> i & 1]
        for a in members:
            add = ns & ~(1 << a) & ~nb[a]
            fill += bin(add).count("1")
            nb[a] |= ns & ~(1 << a)
        alive &= ~(1 << p)
    return fill // 2


def min_fill_exhaustive(adj) -> int:
    n = len(adj)
    return min(fill_of_order(adj, o) for o in itertools.permutations(range(n)))


def md_keyed_brute(adj, verts, key):
    """Minimum degree on the subgraph induced by verts, written from the rule
    itself: at every step recompute every alive vertex's degree in the current
    elimination graph and take the smallest (degree, key, id)."""
    vs = list(verts)
    S = set(vs)
    nb = {v: {u for u in adj[v] if u in S} for v in vs}
    k = dict(zip(vs, key))
    alive = set(vs)
    order = []
    while alive:
        p = min(alive, key=lambda v: (len(nb[v] & alive), k[v], v))
        order.append(p)
        alive.discard(p)
        ns = nb[p] & alive
        for a in ns:
            nb[a] |= ns - {a}
    return order


def leaf_fill_brute(adj, leaf_order):
    """Sum of the column counts of the leaf's columns: eliminate the leaf's
    vertices in order on the graph of the leaf plus its outside neighbours
    (which are never eliminated); each column counts itself and its
    neighbours at elimination time."""
    L = list(leaf_order)
    outside = {u for v in L for u in adj[v]} - set(L)
    S = set(L) | outside
    nb = {v: {u for u in adj[v] if u in S} for v in S}
    alive = set(S)
    total = 0
    for p in L:
        ns = nb[p] & alive - {p}
        total += len(ns) + 1
        alive.discard(p)
        for a in ns:
            nb[a] |= ns - {a}
    return total
