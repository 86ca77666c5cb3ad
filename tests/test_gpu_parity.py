"""GPU path vs the CPU oracle, element by element, through the C ABI.

All outputs are integer: the graph (CSR), the group map (patch per vertex), the
nested-dissection tree (node of every vertex, node begin/size), the
permutation and its inverse, the elimination tree and the column counts must
be bit-exact, at small sizes spanning many patches and tree levels and at the
full benchmark sizes."""
import ctypes

import numpy as np
import pytest
import torch

import meshgen as M
import oracle as O
import paper_2602_00898_b300 as fp

pytestmark = pytest.mark.gpu

_cache = {}


def oracle_all(mesh, cap, seed=0, schedule=0, nd_level=0, lloyd=2):
    key = (mesh.name, mesh.n, mesh.faces.tobytes()[:64], mesh.n_faces, cap, seed, schedule, nd_level, lloyd)
    if key not in _cache:
        g = O.graph_from_faces(mesh.faces, mesh.n)
        o = O.order(g, cap, seed=seed, lloyd_rounds=lloyd, nd_level=nd_level, schedule=schedule)
        s = O.symbolic(g, o.perm)
        _cache[key] = (g, o, s)
    return _cache[key]


def gpu_order(mesh, cap, seed=0, schedule=0, nd_level=0, lloyd=2, dof=1):
    faces = torch.from_numpy(np.ascontiguousarray(mesh.faces)).cuda()
    return fp.order_faces(faces, mesh.n, patch_cap=cap, seed=seed, schedule=schedule, nd_level=nd_level,
                          lloyd_rounds=lloyd, dof_per_vertex=dof)


def np_(t):
    return t.cpu().numpy()


def assert_parity(r, o, s):
    assert r.k == o.k
    np.testing.assert_array_equal(np_(r.gmap), o.label)
    assert r.depth == o.depth
    np.testing.assert_array_equal(np_(r.node_of), o.node_of)
    np.testing.assert_array_equal(np_(r.node_size), o.node_size)
    np.testing.assert_array_equal(np_(r.node_begin), o.node_begin)
    np.testing.assert_array_equal(np_(r.perm), o.perm)
    np.testing.assert_array_equal(np_(r.iperm), o.iperm)
    np.testing.assert_array_equal(np_(r.parent), s.parent)
    np.testing.assert_array_equal(np_(r.colcount), s.colcount)
    assert (r.nnzL, r.flops) == (s.nnzL, s.flops)


def _disconnected_mesh():
    a = M.shuffle(M.torus(12, 10, 0.3, 1), 1)
    b = M.icosphere(2)
    f = np.concatenate([a.faces, b.faces + a.n])
    return M.Mesh("union", a.n + b.n + 5, f.astype(np.int32))


@pytest.mark.parametrize("seed", range(5))
def test_grid64_parity(seed):
    mesh = M.grid64(seed)
    g, o, s = oracle_all(mesh, 256, seed)
    assert_parity(gpu_order(mesh, 256, seed), o, s)


@pytest.mark.parametrize("mesh,cap,seed,kw", [
    (M.shuffle(M.icosphere(4), 3), 100, 3, {}),
    (M.shuffle(M.torus(40, 30, 0.3, 2), 2), 37, 2, {}),
    (_disconnected_mesh(), 50, 4, {}),
    (M.shuffle(M.grid(12, 11), 3), 1, 3, {}),                  # every patch a vertex: classical ND
    (M.shuffle(M.grid(30, 20), 5), 64, 5, {"schedule": 1}),    # level-order schedule
    (M.shuffle(M.grid(30, 20), 6), 64, 6, {"nd_level": 3}),    # leaves hold several patches
    (M.shuffle(M.torus(25, 25, 0.3, 7), 7), 80, 7, {"lloyd": 0}),
    (M.shuffle(M.icosphere(5), 8), 1000, 8, {}),               # separators above 512 vertices
])
def test_small_mesh_parity(mesh, cap, seed, kw):
    g, o, s = oracle_all(mesh, cap, seed, **kw)
    assert_parity(gpu_order(mesh, cap, seed, **kw), o, s)


def test_single_patch_parity():
    mesh = M.shuffle(M.grid(9, 8), 4)
    for seed in range(200):
        g, o, s = oracle_all(mesh, 10**6, seed)
        if o.k == 1:
            break
    assert o.k == 1
    assert_parity(gpu_order(mesh, 10**6, seed), o, s)


def test_isolated_and_empty():
    iso = M.Mesh("iso", 7, np.zeros((0, 3), np.int32))
    g, o, s = oracle_all(iso, 16, 1)
    assert_parity(gpu_order(iso, 16, 1), o, s)
    deg = M.Mesh("degenerate", 6, np.array([[0, 1, 1], [2, 2, 2], [0, 1, 3], [3, 4, 0]], np.int32))
    g, o, s = oracle_all(deg, 2, 0)
    assert_parity(gpu_order(deg, 2, 0), o, s)
    empty = M.Mesh("empty", 0, np.zeros((0, 3), np.int32))
    r = gpu_order(empty, 16)
    assert r.perm.numel() == 0 and r.nnzL == 0


def test_graph_parity_full_sizes():
    for mesh in (M.icosphere7(0), M.torus1024(0)):
        g = O.graph_from_faces(mesh.faces, mesh.n)
        faces = torch.from_numpy(mesh.faces).cuda()
        h = fp.fp_create_from_faces(faces, mesh.n, fp.fp_default_options())
        try:
            n, b, nnz = fp.fp_get_sizes(h)
            assert (n, nnz) == (g.n, g.col.size)
            rp = torch.empty(n + 1, dtype=torch.int32, device="cuda")
            col = torch.empty(nnz, dtype=torch.int32, device="cuda")
            fp.fp_get_graph(h, rp, col)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(np_(rp), g.rowptr)
            np.testing.assert_array_equal(np_(col), g.col)
        finally:
            fp.fp_destroy(h)


def test_icosphere7_full_parity():
    """The benchmark workload (163,842 vertices, cap 512), bit-exact."""
    mesh = M.icosphere7(0)
    g, o, s = oracle_all(mesh, 512, 0)
    assert_parity(gpu_order(mesh, 512, 0), o, s)


def test_torus1024_dof3_full_parity():
    """1024x1024 flipped torus, 3 DOF per vertex: ordering of the vertex graph
    expanded to 3,145,728 unknowns (Section 6.5)."""
    mesh = M.torus1024(0)
    g, o, s = oracle_all(mesh, 512, 0)
    r = gpu_order(mesh, 512, 0, dof=3)
    pd, ad, cd = O.dof_expand(3, o.perm, s.parent, s.colcount)
    np.testing.assert_array_equal(np_(r.perm), pd)
    ipd = np.empty_like(pd); ipd[pd] = np.arange(pd.size, dtype=np.int32)
    np.testing.assert_array_equal(np_(r.iperm), ipd)
    np.testing.assert_array_equal(np_(r.parent), ad)
    np.testing.assert_array_equal(np_(r.colcount), cd)
    assert r.nnzL == 9 * s.nnzL - 3 * g.n
    assert r.nnzL == int(cd.astype(np.int64).sum())
    assert r.flops == int((cd.astype(np.int64) ** 2).sum())
    np.testing.assert_array_equal(np_(r.node_of), o.node_of)
    np.testing.assert_array_equal(np_(r.gmap), o.label)


def _csr_tensors(rows):
    rp = np.cumsum([0] + [len(r) for r in rows]).astype(np.int32)
    col = np.array([c for r in rows for c in r], np.int32)
    return torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda()


def test_csr_scalar_and_block_paths():
    mesh = M.shuffle(M.torus(30, 22, 0.3, 9), 9)
    g, o, s = oracle_all(mesh, 60, 9)
    n = g.n
    # scalar pattern G + I with shuffled column order and duplicates
    rng = np.random.default_rng(0)
    rows = []
    for v in range(n):
        r = list(g.neighbors(v)) + [v, int(g.neighbors(v)[0])]
        rng.shuffle(r)
        rows.append(r)
    rp, col = _csr_tensors(rows)
    r = fp.order_csr(rp, col, n, patch_cap=60, seed=9)
    assert_parity(r, o, s)
    # 3x3 block pattern of the same graph
    b = 3
    brows = [[b * u + c for u in list(g.neighbors(i // b)) + [i // b] for c in range(b)] for i in range(n * b)]
    rp, col = _csr_tensors(brows)
    r = fp.order_csr(rp, col, n * b, patch_cap=60, seed=9, dof_per_vertex=b)
    pd, ad, cd = O.dof_expand(b, o.perm, s.parent, s.colcount)
    np.testing.assert_array_equal(np_(r.perm), pd)
    np.testing.assert_array_equal(np_(r.parent), ad)
    np.testing.assert_array_equal(np_(r.colcount), cd)
    assert r.nnzL == b * b * s.nnzL - n * b * (b - 1) // 2


def test_errors():
    bad = torch.tensor([[0, 1, 7]], dtype=torch.int32, device="cuda")
    with pytest.raises(fp.FpError) as e:
        fp.fp_create_from_faces(bad, 5)
    assert e.value.status == 1
    rp = torch.tensor([0, 1, 1], dtype=torch.int32, device="cuda")
    col = torch.tensor([1], dtype=torch.int32, device="cuda")
    with pytest.raises(fp.FpError) as e:
        fp.fp_create_from_csr(rp, col, 2)
    assert e.value.status == 2
    mesh = M.grid64(0)
    faces = torch.from_numpy(mesh.faces).cuda()
    h = fp.fp_create_from_faces(faces, mesh.n)
    try:
        with pytest.raises(fp.FpError) as e:
            fp.fp_symbolic(h)
        assert e.value.status == 6
    finally:
        fp.fp_destroy(h)


def test_repeatable_bytes():
    mesh = M.shuffle(M.icosphere(5), 11)
    a = gpu_order(mesh, 300, 11)
    b = gpu_order(mesh, 300, 11)
    for x, y in [(a.perm, b.perm), (a.parent, b.parent), (a.colcount, b.colcount), (a.gmap, b.gmap)]:
        assert torch.equal(x, y)


def test_host_buffer_entry_point():
    mesh = M.grid64(3)
    g, o, s = oracle_all(mesh, 256, 3)
    n = mesh.n
    faces = torch.from_numpy(mesh.faces).pin_memory()
    outs = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in range(4)]
    nnz, fl = fp.fp_order_faces_host(faces, n, fp.fp_default_options(patch_cap=256, seed=3), None, *outs)
    np.testing.assert_array_equal(outs[0].numpy(), o.perm)
    np.testing.assert_array_equal(outs[1].numpy(), o.iperm)
    np.testing.assert_array_equal(outs[2].numpy(), s.parent)
    np.testing.assert_array_equal(outs[3].numpy(), s.colcount)
    assert (nnz, fl) == (s.nnzL, s.flops)


def test_host_buffer_entry_point_dof3():
    """The host-buffer form with 3 DOF per vertex (the end-to-end benchmark's
    call): perm and iperm come back while the symbolic factorisation runs."""
    mesh = M.shuffle(M.torus(120, 90, 0.3, 8), 8)
    g, o, s = oracle_all(mesh, 512, 0)
    n, N = mesh.n, 3 * mesh.n
    pd, ad, cd = O.dof_expand(3, o.perm, s.parent, s.colcount)
    ipd = np.empty_like(pd)
    ipd[pd] = np.arange(N, dtype=np.int32)
    faces = torch.from_numpy(mesh.faces).pin_memory()
    for _ in range(2):
        outs = [torch.full((N,), -1, dtype=torch.int32).pin_memory() for _ in range(4)]
        nnz, fl = fp.fp_order_faces_host(faces, n, fp.fp_default_options(patch_cap=512, dof_per_vertex=3), None,
                                         *outs)
        np.testing.assert_array_equal(outs[0].numpy(), pd)
        np.testing.assert_array_equal(outs[1].numpy(), ipd)
        np.testing.assert_array_equal(outs[2].numpy(), ad)
        np.testing.assert_array_equal(outs[3].numpy(), cd)
        assert nnz == 9 * s.nnzL - 3 * n


def _sym_rows(n, edges):
    adj = [set() for _ in range(n)]
    for u, v in edges:
        if u != v:
            adj[u].add(v)
            adj[v].add(u)
    return [sorted(a) for a in adj]


def _dense_random(n, p, seed):
    rng = np.random.default_rng(seed)
    m = np.triu(rng.random((n, n)) < p, 1)
    edges = list(zip(*np.nonzero(m)))
    edges += [(i, i + 1) for i in range(n - 1)]          # connected
    return _sym_rows(n, edges)


# single = one patch, hence one leaf of n vertices and no dissection (checked
# on the oracle: the seeds are drawn by a hash threshold, so the cap alone
# does not fix the patch count)
@pytest.mark.parametrize("kind,n,cap,seed,single", [
    ("clique", 200, 512, 0, True),
    ("dense", 33, 1 << 20, 0, True), ("dense", 63, 1 << 20, 0, True), ("dense", 64, 1 << 20, 0, True),
    ("dense", 65, 1 << 20, 0, True), ("dense", 129, 512, 5, True), ("dense", 512, 1 << 20, 0, True),
    ("star", 300, 1024, 7, True),
    ("chords", 512, 1 << 20, 0, True),
    ("medium", 500, 128, 9, False), ("medium", 400, 96, 10, False),
    ("medium", 2000, 128, 12, False), ("medium", 3000, 128, 13, False),
])
def test_adversarial_graphs_parity(kind, n, cap, seed, single):
    """Leaves up to the 512-vertex limit with pivot rows of up to 16 non-zero
    words and hundreds of neighbours, the 64-vertex padding boundaries of the
    degree scan, a hub of degree n-1, and dense separators whose adjacency
    lists outgrow the separator kernel (global-row fallback: the 570-vertex
    separator of the 3000-vertex graph)."""
    rng = np.random.default_rng(seed)
    if kind == "clique":
        rows = [[u for u in range(n) if u != v] for v in range(n)]
    elif kind == "dense":
        rows = _dense_random(n, 0.3, seed)
    elif kind == "medium":
        rows = _dense_random(n, 20.0 / n, seed)   # mean degree ~20: patch cross edges within capacity
    elif kind == "star":
        rows = _sym_rows(n, [(0, v) for v in range(1, n)])
    else:
        rows = _sym_rows(n, [(i, i + 1) for i in range(n - 1)] +
                         [tuple(rng.integers(0, n, 2)) for _ in range(n // 2)])
    rp, col = _csr_tensors(rows)
    g = O.graph_from_pattern(np_(rp), np_(col))
    o = O.order(g, cap, seed=seed)
    assert (o.k == 1) == single
    s = O.symbolic(g, o.perm)
    r = fp.order_csr(rp, col, n, patch_cap=cap, seed=seed)
    assert_parity(r, o, s)


def test_quotient_capacity_error():
    """A patch with more than 4096 cross-patch edges (a 30%-dense 512-vertex
    graph cut into two patches) is outside the quotient-graph kernel's
    capacity: the call fails with FP_ERR_UNSUPPORTED before any ordering
    kernel runs, and the handle is left unusable."""
    rows = _dense_random(512, 0.3, 6)
    rp, col = _csr_tensors(rows)
    g = O.graph_from_pattern(np_(rp), np_(col))
    assert O.order(g, 512, seed=6).k == 2
    with pytest.raises(fp.FpError) as e:
        fp.order_csr(rp, col, 512, patch_cap=512, seed=6)
    assert fp.STATUS[e.value.status] == "FP_ERR_UNSUPPORTED" and "cross edges" in str(e.value)


def _oracle_given(g, label, k, **kw):
    o = O.order_given(g, label, k, **kw)
    return o, O.symbolic(g, o.perm)


@pytest.mark.parametrize("case", ["computed", "scattered", "empty_labels", "one_group_large", "strips4", "strips2"])
def test_supplied_patches_parity(case):
    """fp_set_patches (Section 4, opening: the patch partition may be
    supplied) against the oracle's order_given: the method's own patches,
    scattered disconnected groups, labels no vertex carries (empty groups),
    one group of 4,096 vertices (a single separator-kernel node), and strips
    of an unshuffled 100x100 grid: four (leaves of ~2,400 vertices, separator
    kernel) and two (leaves of ~4,900, global-row kernel)."""
    if case in ("computed", "scattered", "empty_labels"):
        mesh = M.shuffle(M.torus(30, 22, 0.3, 9), 9)
    elif case == "one_group_large":
        mesh = M.grid64(1)
    else:
        mesh = M.grid(100, 100)        # unshuffled: index ranges are strips of rows
    g = O.graph_from_faces(mesh.faces, mesh.n)
    n = g.n
    if case == "computed":
        oc = O.order(g, 60, seed=9)
        label, k = oc.label, oc.k
    elif case == "scattered":
        label, k = (np.arange(n) * 7919 % 13).astype(np.int32), 13
    elif case == "empty_labels":
        label = (np.arange(n) * 104729 % 40).astype(np.int32)
        label[label % 3 == 1] = 0                 # labels 1, 4, 7, ... left empty
        k = 40
    elif case == "one_group_large":
        label, k = np.zeros(n, np.int32), 1
    else:
        k = 4 if case == "strips4" else 2
        label = (np.arange(n) * k // n).astype(np.int32)
    o, s = _oracle_given(g, label, k)
    faces = torch.from_numpy(np.ascontiguousarray(mesh.faces)).cuda()
    r = fp.order_faces(faces, mesh.n, gmap=torch.from_numpy(np.ascontiguousarray(label, np.int32)).cuda(), k=k)
    assert_parity(r, o, s)


def test_supplied_patches_errors_and_reuse():
    mesh = M.grid(64, 64)                  # unshuffled: index ranges are strips of rows
    faces = torch.from_numpy(np.ascontiguousarray(mesh.faces)).cuda()
    h = fp.fp_create_from_faces(faces, mesh.n)
    try:
        bad = torch.full((mesh.n,), 5, dtype=torch.int32, device="cuda")
        with pytest.raises(fp.FpError) as e:
            fp.fp_set_patches(h, bad, 5)
        assert fp.STATUS[e.value.status] == "FP_ERR_INVALID_ARG"
        with pytest.raises(fp.FpError):
            fp.fp_set_patches(h, bad, 0)
        # the handle stays usable: computed patches, then supplied ones
        perm = torch.empty(mesh.n, dtype=torch.int32, device="cuda")
        fp.fp_permute(h, perm)
        g = O.graph_from_faces(mesh.faces, mesh.n)
        o = O.order(g, 512, seed=0)
        assert np.array_equal(np_(perm), o.perm)
        lab = (np.arange(mesh.n) * 3 // mesh.n).astype(np.int32)
        fp.fp_set_patches(h, torch.from_numpy(lab).cuda(), 3)
        fp.fp_permute(h, perm)
        assert np.array_equal(np_(perm), O.order_given(g, lab, 3).perm)
    finally:
        fp.fp_destroy(h)


def test_csr_bad_row_pointers_rejected():
    """Row pointers that do not start at 0 or that decrease are rejected
    before any column is read through them."""
    L = fp.lib()
    o = fp.fp_default_options()
    col = torch.tensor([1, 0, 2, 1], dtype=torch.int32, device="cuda")
    h = ctypes.c_void_p()
    for bad in ([0, 1, 3, 2], [1, 1, 3, 4], [0, 3, 1, 4]):
        rp = torch.tensor(bad, dtype=torch.int32, device="cuda")
        st = L.fp_create_from_csr(rp.data_ptr(), col.data_ptr(), 3, ctypes.byref(o), None, ctypes.byref(h))
        assert st == 1 and not h.value, bad
        assert "row pointers" in fp.fp_last_error(None)
    rp = torch.tensor([0, 1, 3, 4], dtype=torch.int32, device="cuda")
    assert L.fp_create_from_csr(rp.data_ptr(), None, 3, ctypes.byref(o), None, ctypes.byref(h)) == 1
    assert L.fp_create_from_csr(rp.data_ptr(), col.data_ptr(), 3, ctypes.byref(o), None, ctypes.byref(h)) == 0
    fp.fp_destroy(h)
