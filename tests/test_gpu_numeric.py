"""Numeric factorisation on the GPU (the solver the permutation feeds,
Section 6) against the oracle's up-looking FP64 Cholesky of the same
permuted matrix: the factor column by column and the solutions.

Tolerance: both factorisations are backward stable and the matrices (graph
Laplacians plus the identity, weights in [0.5, 1.5]) have condition numbers
below 2 * max degree * 1.5 + 1 < 40, so forward differences stay near
cond * n_terms * 2^-53 < 1e-12 relative; the tests allow 1e-10 of each
column's largest entry. Where L is structurally zero the GPU value must be
exactly 0.0 (its panel solves by substitution, so no rounding residue
appears there)."""
import ctypes

import numpy as np
import pytest
import torch

import meshgen
import oracle as O

pytestmark = pytest.mark.gpu

RTOL = 1e-10


def _fp():
    import paper_2602_00898_b300 as fp
    return fp


def _factor_both(mesh, cap, wseed, schedule=0, seed=0):
    fp = _fp()
    faces = torch.from_numpy(mesh.faces).cuda()
    h = fp.fp_create_from_faces(faces, mesh.n, fp.fp_default_options(patch_cap=cap, schedule=schedule, seed=seed))
    try:
        perm = torch.empty(mesh.n, dtype=torch.int32, device="cuda")
        fp.fp_permute(h, perm)
        _, _, nnz = fp.fp_get_sizes(h)
        rp = torch.empty(mesh.n + 1, dtype=torch.int32, device="cuda")
        col = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
        fp.fp_get_graph(h, rp, col)
        rpn, coln = rp.cpu().numpy(), col.cpu().numpy()[:nnz]
        diag, off = meshgen.laplacian_values(rpn, coln, seed=wseed)
        fp.fp_factor(h, torch.from_numpy(diag).cuda(), torch.from_numpy(off).cuda())
        cp, ri, rx = fp.fp_factor_export(h)
        rng = np.random.default_rng(17)
        b = rng.standard_normal(mesh.n)
        x = fp.fp_solve(h, torch.from_numpy(b).cuda())
        got = (cp.cpu().numpy(), ri.cpu().numpy(), rx.cpu().numpy(), x.cpu().numpy(), perm.cpu().numpy())
    finally:
        fp.fp_destroy(h)
    g = O.Graph(rpn, coln)
    return got, g, diag, off, b


def _check_factor(got, g, diag, off, b):
    cp, ri, rx, x, perm = got
    n = g.n
    f = O.cholesky(g, diag, off, perm)
    # keys (column, row) of both factors, each sorted
    gk = np.repeat(np.arange(n, dtype=np.int64), np.diff(cp)) * n + ri
    ok = np.repeat(np.arange(n, dtype=np.int64), np.diff(f.Lp)) * n + f.Li
    assert np.all(np.diff(gk) > 0) and np.all(np.diff(ok) > 0)
    at = np.searchsorted(gk, ok)
    assert np.all(at < gk.size) and np.array_equal(gk[at], ok), "a structural nonzero is missing on the GPU"
    colmax = np.zeros(n)
    np.maximum.at(colmax, np.repeat(np.arange(n), np.diff(f.Lp)), np.abs(f.Lx))
    err = np.abs(rx[at] - f.Lx) / colmax[np.repeat(np.arange(n), np.diff(f.Lp))]
    assert err.max() <= RTOL, err.max()
    extra = np.ones(gk.size, bool)
    extra[at] = False
    assert np.all(rx[extra] == 0.0), "nonzero where L is structurally zero"
    # solve: residual and agreement with the oracle's solve
    src = np.repeat(np.arange(n), np.diff(g.rowptr))
    Ax = diag * x + np.bincount(src, weights=off * x[g.col], minlength=n)
    assert np.linalg.norm(Ax - b) <= 1e-12 * np.linalg.norm(b)
    xo = O.cholesky_solve(f, perm, b)
    assert np.abs(x - xo).max() <= 1e-10 * np.abs(xo).max()


@pytest.mark.parametrize("name", ["grid64_unit", "grid64_w", "ico4", "torus48", "grid7x5", "disconnected"])
def test_factor_matches_oracle(name):
    cases = {
        "grid64_unit": (meshgen.grid64(0), 256, None),
        "grid64_w": (meshgen.grid64(2), 64, 4),
        "ico4": (meshgen.shuffle(meshgen.icosphere(4), 2), 128, 5),
        "torus48": (meshgen.shuffle(meshgen.torus(48, 40, 0.3, 5), 5), 200, 6),
        "grid7x5": (meshgen.shuffle(meshgen.grid(7, 5), 1), 4, 7),
        "disconnected": (_disconnected(), 40, 8),
    }
    mesh, cap, w = cases[name]
    _check_factor(*_factor_both(mesh, cap, w))


def _disconnected():
    a = meshgen.shuffle(meshgen.torus(20, 14, 0.3, 1), 1)
    b = meshgen.shuffle(meshgen.icosphere(3), 4)
    f = np.concatenate([a.faces, b.faces + a.n]).astype(np.int32)
    return meshgen.Mesh("union", a.n + b.n + 5, f)


def test_factor_level_order_schedule():
    _check_factor(*_factor_both(meshgen.shuffle(meshgen.icosphere(4), 3), 100, 9, schedule=1, seed=3))


@pytest.mark.slow
def test_factor_icosphere7_full():
    """The 163,842-vertex icosphere (cap 512), every column of L against the
    oracle's factor."""
    _check_factor(*_factor_both(meshgen.icosphere7(0), 512, 1))


def test_factor_errors():
    fp = _fp()
    mesh = meshgen.grid64(0)
    faces = torch.from_numpy(mesh.faces).cuda()
    L = fp.lib()
    h = fp.fp_create_from_faces(faces, mesh.n, fp.fp_default_options(patch_cap=256))
    try:
        b = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
        assert L.fp_solve(h, b.data_ptr(), b.data_ptr()) == 6          # no factor yet
        fp.fp_permute(h)
        _, _, nnz = fp.fp_get_sizes(h)
        diag = torch.ones(mesh.n, dtype=torch.float64, device="cuda")
        off = torch.full((nnz,), -1.0, dtype=torch.float64, device="cuda")
        assert L.fp_factor(h, diag.data_ptr(), off.data_ptr()) == 1     # not positive definite
        assert "positive" in fp.fp_last_error(h)
        assert L.fp_solve(h, b.data_ptr(), b.data_ptr()) == 6
        diag.fill_(7.0)
        assert L.fp_factor(h, diag.data_ptr(), off.data_ptr()) == 0     # the handle is still usable
    finally:
        fp.fp_destroy(h)
    h = fp.fp_create_from_faces(faces, mesh.n, fp.fp_default_options(patch_cap=256, dof_per_vertex=3))
    try:
        fp.fp_permute(h)
        assert L.fp_factor(h, diag.data_ptr(), off.data_ptr()) == 7     # scalar matrices only
    finally:
        fp.fp_destroy(h)
