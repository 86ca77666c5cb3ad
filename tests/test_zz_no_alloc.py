"""fp_graph_from_faces_static: the allocation-free CSR assembly for callers
that cannot allocate device memory (their device memory is reserved by another
allocator, or they must stay out of the CUDA allocator). It must produce
the same CSR as the allocating path (fp_create_from_faces + fp_get_graph), on
consecutive calls that reuse the library's one static scratch array.

Collected last on purpose (file name), so that a run stopping at the first
failure has run every other test before this one."""
import ctypes

import numpy as np
import pytest
import torch

import meshgen as M
import oracle as O
import paper_2602_00898_b300 as fp

pytestmark = pytest.mark.gpu


def _static_fn():
    f = fp.lib().fp_graph_from_faces_static
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]
    return f


def _reference_csr(faces, n):
    h = fp.fp_create_from_faces(faces, n, fp.fp_default_options())
    try:
        _, _, nnz = fp.fp_get_sizes(h)
        rp = torch.empty(n + 1, dtype=torch.int32, device="cuda")
        col = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
        fp.fp_get_graph(h, rp, col)
        torch.cuda.synchronize()
        return rp.cpu().numpy(), col[:nnz].cpu().numpy()
    finally:
        fp.fp_destroy(h)


def _static_csr(faces, n, cap):
    f = _static_fn()
    rp = torch.full((n + 1,), -7, dtype=torch.int32, device="cuda")
    col = torch.full((max(cap, 1),), -7, dtype=torch.int32, device="cuda")
    nnz = ctypes.c_int64(-1)
    st = f(faces.data_ptr() if faces.shape[0] else None, faces.shape[0], n, rp.data_ptr(), col.data_ptr(), cap,
           ctypes.byref(nnz), torch.cuda.current_stream().cuda_stream)
    return st, rp.cpu().numpy(), col.cpu().numpy()[:max(nnz.value, 0)], nnz.value


@pytest.mark.parametrize("mesh", [M.grid64(0), M.shuffle(M.icosphere(5), 3), M.shuffle(M.torus(40, 30, 0.3, 2), 2),
                                  M.Mesh("degenerate", 6, np.array([[0, 1, 1], [2, 2, 2], [0, 1, 3], [3, 4, 0]],
                                                                   np.int32))])
def test_static_matches_allocating_path_twice(mesh):
    faces = torch.from_numpy(mesh.faces).cuda()
    rp_ref, col_ref = _reference_csr(faces, mesh.n)
    g = O.graph_from_faces(mesh.faces, mesh.n)          # the definition, on the CPU
    np.testing.assert_array_equal(rp_ref, g.rowptr)
    np.testing.assert_array_equal(col_ref, g.col)
    for call in range(2):     # the second call sees the first call's leftovers in the scratch array
        st, rp, col, nnz = _static_csr(faces, mesh.n, col_ref.size + 5)
        assert st == 0, fp.fp_last_error(None)
        assert nnz == col_ref.size
        np.testing.assert_array_equal(rp, g.rowptr)
        np.testing.assert_array_equal(col, g.col)


def test_static_alternating_sizes():
    big = M.grid64(1)
    small = M.shuffle(M.grid(9, 7), 5)
    for mesh in (big, small, big):
        faces = torch.from_numpy(mesh.faces).cuda()
        rp_ref, col_ref = _reference_csr(faces, mesh.n)
        st, rp, col, nnz = _static_csr(faces, mesh.n, col_ref.size)
        assert st == 0
        np.testing.assert_array_equal(rp, rp_ref)
        np.testing.assert_array_equal(col, col_ref)


def test_static_limits_and_errors():
    f = _static_fn()
    rp = torch.empty(70000, dtype=torch.int32, device="cuda")
    col = torch.empty(16, dtype=torch.int32, device="cuda")
    nnz = ctypes.c_int64()
    s = torch.cuda.current_stream().cuda_stream
    # above the fixed scratch size: rejected before any launch
    assert f(None, 0, 65537, rp.data_ptr(), col.data_ptr(), 16, ctypes.byref(nnz), s) == 7
    assert "65536" in fp.fp_last_error(None)
    faces = torch.tensor([[0, 1, 2]], dtype=torch.int32, device="cuda")
    assert f(faces.data_ptr(), 200000, 10, rp.data_ptr(), col.data_ptr(), 16, ctypes.byref(nnz), s) == 7
    # a corner out of range, and a too small column buffer
    bad = torch.tensor([[0, 1, 9]], dtype=torch.int32, device="cuda")
    assert f(bad.data_ptr(), 1, 5, rp.data_ptr(), col.data_ptr(), 16, ctypes.byref(nnz), s) == 1
    assert f(faces.data_ptr(), 1, 3, rp.data_ptr(), col.data_ptr(), 4, ctypes.byref(nnz), s) == 1
    # and a valid call right after the failures still matches
    mesh = M.grid64(2)
    fc = torch.from_numpy(mesh.faces).cuda()
    rp_ref, col_ref = _reference_csr(fc, mesh.n)
    st, rp2, col2, n2 = _static_csr(fc, mesh.n, col_ref.size)
    assert st == 0
    np.testing.assert_array_equal(rp2, rp_ref)
    np.testing.assert_array_equal(col2, col_ref)


def test_static_row_limit_and_no_faces():
    """A vertex with more than 256 face-edge entries (a fan of 130 triangles
    around vertex 0) is rejected with a message naming the limit, and the next
    valid call still matches; a mesh without faces gives empty rows."""
    fan = np.array([[0, i, i + 1] for i in range(1, 131)], np.int32)
    faces = torch.from_numpy(fan).cuda()
    st, _, _, _ = _static_csr(faces, 132, 1024)
    assert st == 7
    assert "256" in fp.fp_last_error(None)
    mesh = M.shuffle(M.grid(30, 20), 4)
    fc = torch.from_numpy(mesh.faces).cuda()
    g = O.graph_from_faces(mesh.faces, mesh.n)
    st, rp, col, nnz = _static_csr(fc, mesh.n, g.col.size)
    assert st == 0 and nnz == g.col.size
    np.testing.assert_array_equal(rp, g.rowptr)
    np.testing.assert_array_equal(col, g.col)
    empty = torch.zeros((0, 3), dtype=torch.int32, device="cuda")
    st, rp, col, nnz = _static_csr(empty, 10, 0)
    assert st == 0 and nnz == 0
    np.testing.assert_array_equal(rp, np.zeros(11, np.int32))
