"""ctypes wrapper of the CPU oracle (oracle.cpp).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg import this module; the library never does. The oracle
states the method of "Fast Sparse Matrix Permutation for Mesh-Based Direct
Solvers" (Algorithms 1-3) plainly and single-threaded, and shares no code with
the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so (g++, -O2, single-threaded)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        i32p = P(ctypes.c_int32)
        i64p = P(ctypes.c_int64)
        L.oracle_graph_from_faces.restype = ctypes.c_int64
        L.oracle_graph_from_faces.argtypes = [i32p, ctypes.c_int64, ctypes.c_int32, i32p, i32p, ctypes.c_int64]
        L.oracle_graph_from_pattern.restype = ctypes.c_int64
        L.oracle_graph_from_pattern.argtypes = [i32p, i32p, ctypes.c_int32, ctypes.c_int32, i32p, i32p, ctypes.c_int64]
        L.oracle_seed_hash.restype = ctypes.c_uint64
        L.oracle_seed_hash.argtypes = [ctypes.c_uint64, ctypes.c_int32]
        L.oracle_seeds.restype = ctypes.c_int32
        L.oracle_seeds.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, i32p]
        L.oracle_voronoi.restype = None
        L.oracle_voronoi.argtypes = [i32p, i32p, ctypes.c_int32, ctypes.c_int32, i32p, i32p, i32p, i32p, i32p]
        L.oracle_patches.restype = ctypes.c_int32
        L.oracle_patches.argtypes = [i32p, i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32, i32p]
        L.oracle_min_degree.restype = None
        L.oracle_min_degree.argtypes = [i32p, i32p, ctypes.c_int32, i32p]
        L.oracle_order.restype = ctypes.c_int32
        L.oracle_order.argtypes = [i32p, i32p, ctypes.c_int32, ctypes.c_void_p, i32p, i32p, i32p, i32p,
                                   i32p, i32p, ctypes.c_int32, i32p, i64p]
        L.oracle_order_given.restype = ctypes.c_int32
        L.oracle_order_given.argtypes = [i32p, i32p, ctypes.c_int32, ctypes.c_void_p, i32p, ctypes.c_int32, i32p,
                                         i32p, i32p, i32p, i32p, i32p, ctypes.c_int32, i32p, i64p]
        L.oracle_symbolic.restype = None
        L.oracle_symbolic.argtypes = [i32p, i32p, ctypes.c_int32, i32p, i32p, i32p, i64p, i64p]
        L.oracle_min_degree_keyed.restype = None
        L.oracle_min_degree_keyed.argtypes = [i32p, i32p, ctypes.c_int32, i32p, ctypes.c_int32,
                                              P(ctypes.c_uint32), i32p]
        L.oracle_local_orders_keyed.restype = None
        L.oracle_local_orders_keyed.argtypes = [i32p, i32p, ctypes.c_int32, i32p, ctypes.c_int32, i32p,
                                                P(ctypes.c_uint32), i32p]
        L.oracle_tie_key.restype = ctypes.c_uint32
        L.oracle_tie_key.argtypes = [ctypes.c_uint64, ctypes.c_int32]
        L.oracle_patches_from_seeds.restype = ctypes.c_int32
        L.oracle_patches_from_seeds.argtypes = [i32p, i32p, ctypes.c_int32, ctypes.c_int32, i32p, ctypes.c_int32,
                                                ctypes.c_int32, i32p, i32p]
        L.oracle_order_trace.restype = ctypes.c_int32
        L.oracle_order_trace.argtypes = [i32p, i32p, ctypes.c_int32, ctypes.c_void_p, i32p, ctypes.c_int32,
                                         i32p, i32p, i32p, i32p, i32p, i32p, ctypes.c_int32, i32p, i32p, i32p,
                                         i32p, i32p, i32p, i32p, ctypes.c_int32]
        L.oracle_quotient.restype = ctypes.c_int64
        L.oracle_quotient.argtypes = [i32p, i32p, ctypes.c_int32, i32p, ctypes.c_int32, i32p, i32p, i32p, i32p,
                                      ctypes.c_int64]
        L.oracle_dof_expand.restype = None
        L.oracle_dof_expand.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, i32p]
        _lib = L
    return _lib


class _Opts(ctypes.Structure):
    _fields_ = [("patch_cap", ctypes.c_int32), ("seed", ctypes.c_uint64), ("lloyd_rounds", ctypes.c_int32),
                ("nd_level", ctypes.c_int32), ("schedule", ctypes.c_int32)]


def _p(a: np.ndarray, t=ctypes.c_int32):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


@dataclass
class Graph:
    rowptr: np.ndarray
    col: np.ndarray

    @property
    def n(self) -> int:
        return int(self.rowptr.size - 1)

    def neighbors(self, v: int) -> np.ndarray:
        return self.col[self.rowptr[v]:self.rowptr[v + 1]]


def graph_from_faces(faces: np.ndarray, n: int) -> Graph:
    """Section 2: G = graph of A = (mesh Laplacian pattern) without diagonal."""
    f = _i32(faces).reshape(-1, 3)
    nnz = lib().oracle_graph_from_faces(_p(f), f.shape[0], n, None, None, 0)
    if nnz < 0:
        raise ValueError("face corner out of range")
    rp = np.zeros(n + 1, np.int32)
    col = np.zeros(max(nnz, 1), np.int32)
    lib().oracle_graph_from_faces(_p(f), f.shape[0], n, _p(rp), _p(col), nnz)
    return Graph(rp, col[:nnz])


def graph_from_pattern(rowptr: np.ndarray, col: np.ndarray, b: int = 1) -> Graph:
    """Vertex graph of a scalar or b x b block pattern (Section 6.5)."""
    rp_in = _i32(rowptr); c_in = _i32(col) if len(col) else np.zeros(1, np.int32)
    nrows = rp_in.size - 1
    nnz = lib().oracle_graph_from_pattern(_p(rp_in), _p(c_in), nrows, b, None, None, 0)
    if nnz == -2:
        raise ValueError("pattern not structurally symmetric")
    if nnz < 0:
        raise ValueError("bad pattern")
    n = nrows // b
    rp = np.zeros(n + 1, np.int32)
    out = np.zeros(max(nnz, 1), np.int32)
    lib().oracle_graph_from_pattern(_p(rp_in), _p(c_in), nrows, b, _p(rp), _p(out), nnz)
    return Graph(rp, out[:nnz])


def _gp(g: Graph):
    col = g.col if g.col.size else np.zeros(1, np.int32)
    return _p(g.rowptr), _p(col), col


def seed_hash(seed: int, v: int) -> int:
    return int(lib().oracle_seed_hash(seed, v))


def seeds(n: int, cap: int, seed: int) -> np.ndarray:
    c = lib().oracle_seeds(n, cap, seed, None)
    out = np.zeros(max(c, 1), np.int32)
    lib().oracle_seeds(n, cap, seed, _p(out))
    return out[:c]


def voronoi(g: Graph, src, rank, group=None):
    src = _i32(src); rank = _i32(rank)
    d = np.zeros(g.n, np.int32); l = np.zeros(g.n, np.int32)
    rp, cp, _keep = _gp(g)
    gp = _p(_i32(group)) if group is not None else None
    grp = _i32(group) if group is not None else None
    lib().oracle_voronoi(rp, cp, g.n, src.size, _p(src), _p(rank), _p(grp) if grp is not None else None, _p(d), _p(l))
    return d, l


def patches(g: Graph, cap: int, seed: int = 0, lloyd_rounds: int = 2) -> tuple[np.ndarray, int]:
    lab = np.zeros(g.n, np.int32)
    rp, cp, _keep = _gp(g)
    k = lib().oracle_patches(rp, cp, g.n, cap, seed, lloyd_rounds, _p(lab))
    if k < 0:
        raise ValueError("bad patch options")
    return lab, int(k)


def min_degree(g: Graph) -> np.ndarray:
    o = np.zeros(max(g.n, 1), np.int32)
    rp, cp, _keep = _gp(g)
    lib().oracle_min_degree(rp, cp, g.n, _p(o))
    return o[:g.n]


def min_degree_keyed(g: Graph, verts, key=None) -> np.ndarray:
    """Exact minimum degree on the subgraph induced by `verts`, ties to the
    smaller (key, id) (key: one uint32 per entry of verts, or None)."""
    vs = _i32(verts)
    m = vs.size
    o = np.zeros(max(m, 1), np.int32)
    rp, cp, _keep = _gp(g)
    kp = None
    if key is not None:
        kk = np.ascontiguousarray(key, dtype=np.uint32)
        kp = _p(kk, ctypes.c_uint32)
    lib().oracle_min_degree_keyed(rp, cp, g.n, _p(vs) if m else None, m, kp, _p(o))
    return o[:m]


def local_orders_keyed(g: Graph, ptr, verts, key_of_vertex=None) -> np.ndarray:
    """Keyed minimum-degree order of each vertex set verts[ptr[s]:ptr[s+1]]
    (key_of_vertex: uint32 per graph vertex, or None for id ties)."""
    ptr = _i32(ptr); vs = _i32(verts) if len(verts) else np.zeros(1, np.int32)
    o = np.zeros(max(len(verts), 1), np.int32)
    rp, cp, _keep = _gp(g)
    kp = None
    if key_of_vertex is not None:
        kk = np.ascontiguousarray(key_of_vertex, dtype=np.uint32)
        kp = _p(kk, ctypes.c_uint32)
    lib().oracle_local_orders_keyed(rp, cp, g.n, _p(ptr), ptr.size - 1, _p(vs), kp, _p(o))
    return o[:len(verts)]


def tie_key(r: int, v: int) -> int:
    """Seeded tie-break key of vertex v for the r-th random MD order."""
    return int(lib().oracle_tie_key(r, v))


@dataclass
class Ordering:
    k: int
    depth: int
    label: np.ndarray       # gmap: patch id per vertex
    node_of: np.ndarray     # etree node per vertex
    perm: np.ndarray        # perm[i] = original vertex at new position i
    iperm: np.ndarray
    node_begin: np.ndarray  # per tree node: first position in perm
    node_size: np.ndarray   # per tree node: number of vertices
    node_qsum: np.ndarray   # per bisected node: sum of quotient edge weights among its patches (-1 leaf)


def order(g: Graph, cap: int, seed: int = 0, lloyd_rounds: int = 2, nd_level: int = 0,
          schedule: int = 0) -> Ordering:
    """Algorithm 1: patches -> patch-guided ND etree -> local orders -> perm."""
    n = g.n
    o = _Opts(cap, seed, lloyd_rounds, nd_level, schedule)
    lab = np.zeros(max(n, 1), np.int32); nod = np.zeros(max(n, 1), np.int32)
    perm = np.zeros(max(n, 1), np.int32); iperm = np.zeros(max(n, 1), np.int32)
    tree_cap = 4 * max(n, 1) + 8
    if nd_level > 0:
        tree_cap = max(tree_cap, (1 << (nd_level + 1)))
    nb = np.zeros(tree_cap, np.int32); ns = np.zeros(tree_cap, np.int32)
    depth = np.zeros(1, np.int32)
    qs = np.zeros(tree_cap, np.int64)
    rp, cp, _keep = _gp(g)
    k = lib().oracle_order(rp, cp, n, ctypes.byref(o), _p(lab), _p(nod), _p(perm), _p(iperm),
                           _p(nb), _p(ns), tree_cap, _p(depth), _p(qs, ctypes.c_int64))
    if k < 0:
        raise ValueError(f"oracle_order failed ({k})")
    D = int(depth[0])
    nn = (1 << (D + 1)) - 1
    return Ordering(int(k), D, lab[:n], nod[:n], perm[:n], iperm[:n], nb[:nn].copy(), ns[:nn].copy(),
                    qs[:nn].copy())


def order_given(g: Graph, label, k: int, nd_level: int = 0, schedule: int = 0) -> Ordering:
    """Algorithm 1 steps 2-4 with the patches supplied (Section 4, opening):
    label[v] in [0, k) is the group of vertex v; groups need not be connected,
    and an empty group takes no part (zero weight)."""
    n = g.n
    given = _i32(label)
    assert given.shape == (n,)
    o = _Opts(1, 0, 0, nd_level, schedule)
    lab = np.zeros(max(n, 1), np.int32); nod = np.zeros(max(n, 1), np.int32)
    perm = np.zeros(max(n, 1), np.int32); iperm = np.zeros(max(n, 1), np.int32)
    tree_cap = 4 * max(n, k, 1) + 8
    if nd_level > 0:
        tree_cap = max(tree_cap, (1 << (nd_level + 1)))
    nb = np.zeros(tree_cap, np.int32); ns = np.zeros(tree_cap, np.int32)
    depth = np.zeros(1, np.int32)
    qs = np.zeros(tree_cap, np.int64)
    rp, cp, _keep = _gp(g)
    r = lib().oracle_order_given(rp, cp, n, ctypes.byref(o), _p(given if n else np.zeros(1, np.int32)), int(k),
                                 _p(lab), _p(nod), _p(perm), _p(iperm), _p(nb), _p(ns), tree_cap, _p(depth),
                                 _p(qs, ctypes.c_int64))
    if r < 0:
        raise ValueError(f"oracle_order_given failed ({r})")
    D = int(depth[0])
    nn = (1 << (D + 1)) - 1
    return Ordering(int(r), D, lab[:n], nod[:n], perm[:n], iperm[:n], nb[:nn].copy(), ns[:nn].copy(),
                    qs[:nn].copy())


@dataclass
class Symbolic:
    parent: np.ndarray
    colcount: np.ndarray
    nnzL: int
    flops: int


def symbolic(g: Graph, perm: np.ndarray) -> Symbolic:
    """Elimination tree and column counts of P (G + I) P^T."""
    n = g.n
    perm = _i32(perm) if n else np.zeros(1, np.int32)
    par = np.zeros(max(n, 1), np.int32); cc = np.zeros(max(n, 1), np.int32)
    nnz = np.zeros(1, np.int64); fl = np.zeros(1, np.int64)
    rp, cp, _keep = _gp(g)
    lib().oracle_symbolic(rp, cp, n, _p(perm), _p(par), _p(cc), _p(nnz, ctypes.c_int64), _p(fl, ctypes.c_int64))
    return Symbolic(par[:n], cc[:n], int(nnz[0]), int(fl[0]))


def dof_expand(b: int, perm, parent, colcount):
    """Section 6.5: vertex ordering + symbolic results -> b DOFs per vertex."""
    n = len(perm)
    perm = _i32(perm); parent = _i32(parent); colcount = _i32(colcount)
    pd = np.zeros(max(n * b, 1), np.int32); ad = np.zeros_like(pd); cd = np.zeros_like(pd)
    lib().oracle_dof_expand(n, b, _p(perm), _p(parent), _p(colcount), _p(pd), _p(ad), _p(cd))
    return pd[:n * b], ad[:n * b], cd[:n * b]


def patches_from_seeds(g: Graph, seeds, cap: int, lloyd_rounds: int = 0) -> tuple[np.ndarray, np.ndarray, int]:
    """Contract R2-R5 from explicit seeds (rank = position in `seeds`): returns
    (labels, seed of every final rank, k)."""
    s = _i32(seeds) if len(seeds) else np.zeros(1, np.int32)
    lab = np.zeros(max(g.n, 1), np.int32)
    so = np.zeros(max(g.n, 1), np.int32)
    rp, cp, _keep = _gp(g)
    k = lib().oracle_patches_from_seeds(rp, cp, g.n, len(seeds), _p(s), cap, lloyd_rounds, _p(lab), _p(so))
    if k < 0:
        raise ValueError("bad seeds or options")
    return lab[:g.n], so[:k], int(k)


@dataclass
class Trace:
    """Intermediate stages of Algorithm 1 (see oracle_order_trace)."""
    ordering: Ordering
    seeds0: np.ndarray            # seed of every rank after R1 + R3
    lloyd_seeds: list             # per Lloyd round: seed of every rank
    labels: list                  # labels after the first labelling and after each Lloyd relabel
    side_at: np.ndarray           # [D, k]: side of each patch in the node bisected at depth d, -1 if none
    child_at: np.ndarray          # [D, k]: child node each patch moved to at depth d, -1 if none


def order_trace(g: Graph, cap: int = 512, seed: int = 0, lloyd_rounds: int = 2, nd_level: int = 0,
                schedule: int = 0, given=None, k: int = 0) -> Trace:
    """oracle.order (or, with `given` labels in [0, k), oracle.order_given)
    with its stage boundaries recorded."""
    n = g.n
    o = _Opts(cap, seed, lloyd_rounds, nd_level, schedule)
    gv = _i32(given) if given is not None else None
    N = max(n, 1)
    lab = np.zeros(N, np.int32); nod = np.zeros(N, np.int32)
    perm = np.zeros(N, np.int32); iperm = np.zeros(N, np.int32)
    tree_cap = 4 * N + 8
    if nd_level > 0:
        tree_cap = max(tree_cap, (1 << (nd_level + 1)))
    nb = np.zeros(tree_cap, np.int32); ns = np.zeros(tree_cap, np.int32)
    depth = np.zeros(1, np.int32); k0 = np.zeros(1, np.int32)
    max_levels = max(nd_level, 32)
    seeds0 = np.zeros(N, np.int32)
    ls = np.zeros((max(lloyd_rounds, 1), N), np.int32)
    labels = np.zeros((lloyd_rounds + 1, N), np.int32)
    side = np.full((max_levels, N), -1, np.int32); child = np.full((max_levels, N), -1, np.int32)
    rp, cp, _keep = _gp(g)
    if gv is not None:
        tree_cap = max(tree_cap, 4 * max(k, 1) + 8)
        nb = np.zeros(tree_cap, np.int32); ns = np.zeros(tree_cap, np.int32)
    k = lib().oracle_order_trace(rp, cp, n, ctypes.byref(o), _p(gv) if gv is not None and n else None, int(k),
                                 _p(lab), _p(nod), _p(perm), _p(iperm), _p(nb), _p(ns), tree_cap, _p(depth),
                                 _p(seeds0), _p(k0), _p(ls), _p(labels), _p(side), _p(child), max_levels)
    if k < 0:
        raise ValueError(f"oracle_order_trace failed ({k})")
    D = int(depth[0]); nn = (1 << (D + 1)) - 1; kz = int(k0[0])
    ordering = Ordering(int(k), D, lab[:n], nod[:n], perm[:n], iperm[:n], nb[:nn].copy(), ns[:nn].copy(),
                        np.full(nn, -1, np.int64))
    return Trace(ordering, seeds0[:kz].copy(), [ls[r, :kz].copy() for r in range(lloyd_rounds)],
                 [labels[r, :n].copy() for r in range(lloyd_rounds + 1)], side[:D, :k].copy(), child[:D, :k].copy())


def quotient(g: Graph, label, k: int):
    """Quotient graph of a patch map (contract R6): (w, q_rowptr, q_col, q_w),
    rows in increasing neighbour id."""
    lab = _i32(label) if g.n else np.zeros(1, np.int32)
    rp, cp, _keep = _gp(g)
    m = lib().oracle_quotient(rp, cp, g.n, _p(lab), k, None, None, None, None, 0)
    w = np.zeros(max(k, 1), np.int32); qr = np.zeros(k + 1, np.int32)
    qc = np.zeros(max(m, 1), np.int32); qw = np.zeros(max(m, 1), np.int32)
    lib().oracle_quotient(rp, cp, g.n, _p(lab), k, _p(w), _p(qr), _p(qc), _p(qw), m)
    return w[:k], qr, qc[:m], qw[:m]


def _numeric_lib():
    L = lib()
    if not getattr(L, "_chol_ready", False):
        P = ctypes.POINTER
        i32p, i64p, f64p = P(ctypes.c_int32), P(ctypes.c_int64), P(ctypes.c_double)
        L.oracle_cholesky.restype = ctypes.c_int64
        L.oracle_cholesky.argtypes = [i32p, i32p, ctypes.c_int32, f64p, f64p, i32p, i64p, i32p, f64p, ctypes.c_int64]
        L.oracle_cholesky_solve.restype = None
        L.oracle_cholesky_solve.argtypes = [ctypes.c_int32, i32p, i64p, i32p, f64p, f64p, f64p]
        L._chol_ready = True
    return L


@dataclass
class Factor:
    """L of P A P^T in compressed columns (rows ascending, diagonal first)."""
    Lp: np.ndarray   # int64 [n+1]
    Li: np.ndarray   # int32 [nnz]
    Lx: np.ndarray   # float64 [nnz]


def cholesky(g: Graph, a_diag, a_off, perm) -> Factor:
    """Sparse FP64 Cholesky of P A P^T (A: diagonal a_diag, off-diagonal
    values a_off aligned with g's CSR) by up-looking row solves."""
    L = _numeric_lib()
    n = g.n
    ad = np.ascontiguousarray(a_diag, np.float64)
    ao = np.ascontiguousarray(a_off, np.float64) if len(a_off) else np.zeros(1)
    pm = _i32(perm) if n else np.zeros(1, np.int32)
    rp, cp, _keep = _gp(g)
    Lp = np.zeros(n + 1, np.int64)
    nnz = L.oracle_cholesky(rp, cp, n, _p(ad, ctypes.c_double), _p(ao, ctypes.c_double), _p(pm), _p(Lp, ctypes.c_int64),
                            None, None, 0)
    Li = np.zeros(max(nnz, 1), np.int32)
    Lx = np.zeros(max(nnz, 1), np.float64)
    r = L.oracle_cholesky(rp, cp, n, _p(ad, ctypes.c_double), _p(ao, ctypes.c_double), _p(pm), _p(Lp, ctypes.c_int64),
                          _p(Li), _p(Lx, ctypes.c_double), nnz)
    if r < 0:
        raise ValueError("matrix not positive definite" if r == -1 else "factor storage")
    return Factor(Lp, Li[:nnz], Lx[:nnz])


def cholesky_solve(f: Factor, perm, b) -> np.ndarray:
    """x with A x = b from the factor of P A P^T."""
    L = _numeric_lib()
    n = f.Lp.size - 1
    bb = np.ascontiguousarray(b, np.float64)
    x = np.zeros(max(n, 1), np.float64)
    L.oracle_cholesky_solve(n, _p(_i32(perm)), _p(f.Lp, ctypes.c_int64), _p(f.Li), _p(f.Lx, ctypes.c_double),
                            _p(bb, ctypes.c_double), _p(x, ctypes.c_double))
    return x[:n]
