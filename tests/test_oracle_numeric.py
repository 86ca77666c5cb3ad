"""Pins of the oracle's numeric factorisation (the solver the permutation and
its elimination tree drive, Section 6): a hand-computed factor, the dense
LAPACK Cholesky of the same permuted matrix, the symbolic column counts and
solve residuals."""
from __future__ import annotations

import math

import numpy as np
import pytest

import meshgen as M
import oracle as O


def _dense(g, diag, off):
    n = g.n
    A = np.zeros((n, n))
    src = np.repeat(np.arange(n), np.diff(g.rowptr))
    A[src, g.col] = off
    A[np.arange(n), np.arange(n)] = diag
    return A


def _dense_L(f, n):
    L = np.zeros((n, n))
    for j in range(n):
        L[f.Li[f.Lp[j]:f.Lp[j + 1]], j] = f.Lx[f.Lp[j]:f.Lp[j + 1]]
    return L


def test_hand_computed_factor_of_a_path():
    # A = [[2,-1,0],[-1,3,-1],[0,-1,2]] in the identity order:
    # L11 = sqrt 2, L21 = -1/sqrt 2, L22 = sqrt(3 - 1/2), L32 = -1/L22,
    # L33 = sqrt(2 - 1/L22^2)
    g = O.Graph(np.array([0, 1, 3, 4], np.int32), np.array([1, 0, 2, 1], np.int32))
    f = O.cholesky(g, [2.0, 3.0, 2.0], [-1.0, -1.0, -1.0, -1.0], [0, 1, 2])
    l22 = math.sqrt(2.5)
    want = [math.sqrt(2), -1 / math.sqrt(2), l22, -1 / l22, math.sqrt(2 - 1 / 2.5)]
    assert f.Lp.tolist() == [0, 2, 4, 5]
    assert f.Li.tolist() == [0, 1, 1, 2, 2]
    assert np.allclose(f.Lx, want, rtol=0, atol=1e-15)
    # the reversed order: eliminating 2 first gives L11 = sqrt 2 at vertex 2
    f2 = O.cholesky(g, [2.0, 3.0, 2.0], [-1.0, -1.0, -1.0, -1.0], [2, 1, 0])
    assert np.allclose(f2.Lx, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", [None, 3])
def test_factor_matches_dense_cholesky_on_grid(seed):
    """64x64 grid (4,096 vertices) in the method's order: the sparse factor
    equals LAPACK's dense Cholesky of P A P^T entry by entry, its residual is
    below 1e-10 relative, and its nonzeros per column are exactly the
    symbolic column counts (a Stieltjes matrix: no cancellation)."""
    m = M.grid64(0)
    g = O.graph_from_faces(m.faces, m.n)
    o = O.order(g, 256)
    diag, off = M.laplacian_values(g.rowptr, g.col, seed=seed)
    f = O.cholesky(g, diag, off, o.perm)
    s = O.symbolic(g, o.perm)
    assert np.array_equal(np.diff(f.Lp), s.colcount)
    A = _dense(g, diag, off)
    B = A[np.ix_(o.perm, o.perm)]
    Ld = np.linalg.cholesky(B)
    L = _dense_L(f, g.n)
    assert np.abs(L - Ld).max() <= 1e-12 * np.abs(Ld).max()
    assert np.abs(L @ L.T - B).max() / np.abs(B).max() <= 1e-10
    # structure: exactly the nonzeros of the dense factor
    assert np.array_equal(L != 0, np.abs(Ld) > 0)
    # every column's rows ascend, diagonal first, and the first off-diagonal
    # row is the elimination-tree parent
    for j in range(0, g.n, 37):
        rows = f.Li[f.Lp[j]:f.Lp[j + 1]]
        assert rows[0] == j and np.all(np.diff(rows) > 0)
        assert (rows[1] if rows.size > 1 else -1) == s.parent[j]


def test_solve_residual():
    m = M.shuffle(M.icosphere(4), 2)
    g = O.graph_from_faces(m.faces, m.n)
    o = O.order(g, 128, seed=2)
    diag, off = M.laplacian_values(g.rowptr, g.col, seed=5)
    f = O.cholesky(g, diag, off, o.perm)
    A = _dense(g, diag, off)
    rng = np.random.default_rng(1)
    for _ in range(3):
        b = rng.standard_normal(g.n)
        x = O.cholesky_solve(f, o.perm, b)
        assert np.linalg.norm(A @ x - b) <= 1e-12 * np.linalg.norm(b)


def test_not_positive_definite_is_reported():
    g = O.Graph(np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32))
    with pytest.raises(ValueError):
        O.cholesky(g, [1.0, 1.0], [-2.0, -2.0], [0, 1])
