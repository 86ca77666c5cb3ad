"""Batched ordering (fp_batch_order / fp_batch_autotune) against the oracle:
every mesh of a batch must come out bit-identical to the oracle run on that
mesh alone with the cap the batch used."""
import numpy as np
import pytest
import torch

import meshgen as M
import oracle as O
import paper_2602_00898_b300 as fp

pytestmark = pytest.mark.gpu


def _mix(count, seed, lo=1500, hi=20000):
    return M.mesh_mix(count, seed, lo, hi)


def _check_item(mesh, it, outs, dof=1):
    assert it.status == 0
    g = O.graph_from_faces(mesh.faces, mesh.n)
    o = O.order(g, it.chosen_cap, seed=0)
    s = O.symbolic(g, o.perm)
    perm, iperm, parent, colcount = [t.cpu().numpy()[:mesh.n * dof] for t in outs]
    if dof == 1:
        np.testing.assert_array_equal(perm, o.perm)
        np.testing.assert_array_equal(iperm, o.iperm)
        np.testing.assert_array_equal(parent, s.parent)
        np.testing.assert_array_equal(colcount, s.colcount)
        assert (it.nnzL, it.flops) == (s.nnzL, s.flops)
    else:
        pd, ad, cd = O.dof_expand(dof, o.perm, s.parent, s.colcount)
        np.testing.assert_array_equal(perm, pd)
        np.testing.assert_array_equal(parent, ad)
        np.testing.assert_array_equal(colcount, cd)
        assert it.nnzL == dof * dof * s.nnzL - mesh.n * dof * (dof - 1) // 2


def test_batch_explicit_caps_matches_oracle():
    meshes = _mix(12, 7)
    caps = [64, 128, 256, 512] * 3
    faces = [torch.from_numpy(m.faces).cuda() for m in meshes]
    items = fp.make_batch(faces, [m.n for m in meshes], caps)
    st = fp.fp_batch_order(items, fp.fp_default_options(), n_workers=5)
    torch.cuda.synchronize()
    assert st == 0
    assert [it.chosen_cap for it in items] == caps
    for m, it, (_, outs) in zip(meshes, items, items.tensors):
        _check_item(m, it, outs)


def test_batch_autotuned_caps():
    meshes = _mix(8, 11, 2000, 60000)
    faces = [torch.from_numpy(m.faces).cuda() for m in meshes]
    items = fp.make_batch(faces, [m.n for m in meshes])
    chosen = fp.fp_batch_autotune(items, fp.fp_default_options())
    assert all(c in (0, 128, 256, 384, 512) for c in chosen) and any(chosen)
    st = fp.fp_batch_order(items, fp.fp_default_options(), n_workers=4)
    torch.cuda.synchronize()
    assert st == 0
    for m, it, (_, outs) in zip(meshes, items, items.tensors):
        assert it.chosen_cap in (128, 256, 384, 512)
        _check_item(m, it, outs)


def test_batch_item_failure_is_isolated():
    meshes = _mix(4, 3)
    faces = [torch.from_numpy(m.faces).cuda() for m in meshes]
    bad = torch.tensor([[0, 1, 999999]], dtype=torch.int32, device="cuda")
    items = fp.make_batch(faces + [bad], [m.n for m in meshes] + [10], [200] * 5)
    st = fp.fp_batch_order(items, fp.fp_default_options(), n_workers=3)
    torch.cuda.synchronize()
    assert st == 1
    assert [it.status for it in items] == [0, 0, 0, 0, 1]
    for m, it, (_, outs) in zip(meshes, list(items)[:4], items.tensors[:4]):
        _check_item(m, it, outs)


def test_batch_dof3():
    meshes = [M.shuffle(M.torus(40, 36, 0.3, s), s) for s in range(3)]
    faces = [torch.from_numpy(m.faces).cuda() for m in meshes]
    items = fp.make_batch(faces, [m.n for m in meshes], [100, 200, 300], dof=3)
    st = fp.fp_batch_order(items, fp.fp_default_options(dof_per_vertex=3), n_workers=3)
    torch.cuda.synchronize()
    assert st == 0
    for m, it, (_, outs) in zip(meshes, items, items.tensors):
        _check_item(m, it, outs, dof=3)


def test_batch_learned_matches_oracle():
    """fp_batch_order_learned: every mesh equals the oracle's learned ordering
    of that mesh alone (same cap, same network), with the same choices."""
    from oracle import gnn as G
    meshes = _mix(6, 19, 1500, 12000)
    caps = [128, 256, 512, 128, 256, 512]
    d = M.gnn_weights(31)
    codes = fp.pack_params(d, np.int32)
    faces = [torch.from_numpy(m.faces).cuda() for m in meshes]
    items = fp.make_batch(faces, [m.n for m in meshes], caps)
    st = fp.fp_batch_order_learned(items, codes, fp.fp_default_options(), n_workers=3)
    torch.cuda.synchronize()
    assert st == 0
    for m, it, (_, outs) in zip(meshes, items, items.tensors):
        g = O.graph_from_faces(m.faces, m.n)
        o = O.order(g, it.chosen_cap, seed=0)
        L = G.order_learned(g, o, G.QParams.from_dict(d), it.chosen_cap)
        s = O.symbolic(g, L.perm)
        perm, iperm, parent, colcount = [t.cpu().numpy()[:m.n] for t in outs]
        np.testing.assert_array_equal(perm, L.perm)
        np.testing.assert_array_equal(parent, s.parent)
        np.testing.assert_array_equal(colcount, s.colcount)
        assert (it.nnzL, it.flops) == (s.nnzL, s.flops)
        assert it.learned_leaves == len(L.leaves) and it.learned_kept == int(L.kept.sum())
        assert it.fill_plain == int(L.fill_plain.sum())
        assert it.fill_chosen == int(np.where(L.kept, L.fill_learned, L.fill_plain).sum())


def test_full_batch_256_sampled():
    """The benchmark's full batch: 256 meshes of 2k-200k vertices with
    autotuned caps. Every 16th mesh is checked bit for bit against the oracle
    run alone with the cap the batch chose; every mesh gets the invariants
    (perm a bijection, iperm its inverse, nnz(L) >= n, a root etree column)."""
    meshes = M.mesh_mix(256, seed=0)
    faces = [torch.from_numpy(m.faces).cuda() for m in meshes]
    items = fp.make_batch(faces, [m.n for m in meshes])
    fp.fp_batch_autotune(items, fp.fp_default_options())
    st = fp.fp_batch_order(items, fp.fp_default_options())
    torch.cuda.synchronize()
    assert st == 0
    for i, (m, it, (_, outs)) in enumerate(zip(meshes, items, items.tensors)):
        assert it.status == 0 and it.nnzL >= m.n
        perm, iperm, parent = [t.cpu().numpy()[:m.n] for t in outs[:3]]
        assert np.array_equal(np.sort(perm), np.arange(m.n))
        assert np.array_equal(iperm[perm], np.arange(m.n))
        assert (parent == -1).any() and ((parent == -1) | (parent > np.arange(m.n))).all()
        if i % 16 == 0:
            _check_item(m, it, outs)


# ---- the fused form (n_workers = 0): the whole batch as one disjoint union ----

def _tiny_meshes():
    """Degenerate members: an empty mesh, one vertex, isolated vertices only, a
    single triangle, and a mesh of two components plus isolated vertices."""
    a = M.shuffle(M.torus(12, 10, 0.3, 1), 1)
    b = M.shuffle(M.icosphere(2), 2)
    two = np.concatenate([a.faces, b.faces + a.n]).astype(np.int32)
    return [M.Mesh("empty", 0, np.zeros((0, 3), np.int32)),
            M.Mesh("one", 1, np.zeros((0, 3), np.int32)),
            M.Mesh("isolated", 9, np.zeros((0, 3), np.int32)),
            M.Mesh("triangle", 3, np.array([[0, 1, 2]], np.int32)),
            M.Mesh("two+isolated", a.n + b.n + 4, two)]


def test_fused_explicit_caps_matches_oracle():
    meshes = _mix(12, 7) + _tiny_meshes()
    caps = [64, 128, 256, 512] * 3 + [16, 16, 4, 2, 40]
    faces = [torch.from_numpy(m.faces).cuda() for m in meshes]
    items = fp.make_batch(faces, [m.n for m in meshes], caps)
    st = fp.fp_batch_order(items, fp.fp_default_options(), n_workers=0)
    torch.cuda.synchronize()
    assert st == 0
    assert [it.chosen_cap for it in items] == caps
    assert items[0].launches > 0 and all(it.launches == 0 for it in list(items)[1:])
    for m, it, (_, outs) in zip(meshes, items, items.tensors):
        _check_item(m, it, outs)


def test_fused_equals_pool():
    """The same batch through the fused union and through the per-mesh pool:
    every output and every count identical."""
    meshes = _mix(20, 23, 1500, 40000)
    faces = [torch.from_numpy(m.faces).cuda() for m in meshes]
    caps = [128, 192, 256, 384, 512] * 4
    a = fp.make_batch(faces, [m.n for m in meshes], caps)
    b = fp.make_batch(faces, [m.n for m in meshes], caps)
    assert fp.fp_batch_order(a, fp.fp_default_options(), n_workers=0) == 0
    assert fp.fp_batch_order(b, fp.fp_default_options(), n_workers=6) == 0
    torch.cuda.synchronize()
    for x, y, (_, ox), (_, oy) in zip(a, b, a.tensors, b.tensors):
        assert (x.nnzL, x.flops, x.chosen_cap, x.status) == (y.nnzL, y.flops, y.chosen_cap, y.status)
        for tx, ty in zip(ox, oy):
            assert torch.equal(tx, ty)


def test_fused_single_mesh_and_seeds():
    """A batch of one mesh, and the seed option reaching every member."""
    m = M.shuffle(M.icosphere(5), 8)
    faces = [torch.from_numpy(m.faces).cuda()]
    items = fp.make_batch(faces, [m.n], [300])
    assert fp.fp_batch_order(items, fp.fp_default_options(), n_workers=0) == 0
    _check_item(m, items[0], items.tensors[0][1])
    meshes = _mix(5, 29)
    faces = [torch.from_numpy(x.faces).cuda() for x in meshes]
    items = fp.make_batch(faces, [x.n for x in meshes], [256] * 5)
    assert fp.fp_batch_order(items, fp.fp_default_options(seed=5, lloyd_rounds=1), n_workers=0) == 0
    torch.cuda.synchronize()
    for x, it, (_, outs) in zip(meshes, items, items.tensors):
        g = O.graph_from_faces(x.faces, x.n)
        o = O.order(g, 256, seed=5, lloyd_rounds=1)
        np.testing.assert_array_equal(outs[0].cpu().numpy(), o.perm)


def test_fused_failure_reports_every_item():
    """A corner outside its own mesh (though inside the union) fails the fused
    pipeline; the items are then ordered one by one and each gets its own
    status."""
    meshes = _mix(4, 3)
    faces = [torch.from_numpy(m.faces).cuda() for m in meshes]
    bad = torch.tensor([[0, 1, 12]], dtype=torch.int32, device="cuda")   # vertex 12 of a 10-vertex mesh
    items = fp.make_batch(faces + [bad], [m.n for m in meshes] + [10], [200] * 5)
    st = fp.fp_batch_order(items, fp.fp_default_options(), n_workers=0)
    torch.cuda.synchronize()
    assert st == 1
    assert [it.status for it in items] == [0, 0, 0, 0, 1]
    for m, it, (_, outs) in zip(meshes, list(items)[:4], items.tensors[:4]):
        _check_item(m, it, outs)


def test_fused_learned_matches_oracle_and_pool():
    """fp_batch_order_learned in the fused form: every mesh equals the oracle's
    learned ordering of that mesh alone, the per-mesh choice statistics match,
    and the pool form gives the same items."""
    from oracle import gnn as G
    meshes = _mix(6, 19, 1500, 12000) + _tiny_meshes()[2:]
    caps = [128, 256, 512, 128, 256, 512, 4, 2, 40]
    d = M.gnn_weights(31)
    codes = fp.pack_params(d, np.int32)
    faces = [torch.from_numpy(m.faces).cuda() for m in meshes]
    items = fp.make_batch(faces, [m.n for m in meshes], caps)
    pool = fp.make_batch(faces, [m.n for m in meshes], caps)
    assert fp.fp_batch_order_learned(items, codes, fp.fp_default_options(), n_workers=0) == 0
    assert fp.fp_batch_order_learned(pool, codes, fp.fp_default_options(), n_workers=4) == 0
    torch.cuda.synchronize()
    for m, it, (_, outs), jt, (_, pouts) in zip(meshes, items, items.tensors, pool, pool.tensors):
        g = O.graph_from_faces(m.faces, m.n)
        o = O.order(g, it.chosen_cap, seed=0)
        L = G.order_learned(g, o, G.QParams.from_dict(d), it.chosen_cap)
        s = O.symbolic(g, L.perm)
        perm, iperm, parent, colcount = [t.cpu().numpy()[:m.n] for t in outs]
        np.testing.assert_array_equal(perm, L.perm)
        np.testing.assert_array_equal(parent, s.parent)
        np.testing.assert_array_equal(colcount, s.colcount)
        assert (it.nnzL, it.flops) == (s.nnzL, s.flops)
        assert it.learned_leaves == len(L.leaves) and it.learned_kept == int(L.kept.sum())
        assert it.fill_plain == int(L.fill_plain.sum())
        assert it.fill_chosen == int(np.where(L.kept, L.fill_learned, L.fill_plain).sum())
        assert (it.learned_leaves, it.learned_kept, it.fill_plain, it.fill_chosen) == \
            (jt.learned_leaves, jt.learned_kept, jt.fill_plain, jt.fill_chosen)
        for tx, ty in zip(outs, pouts):
            assert torch.equal(tx, ty)


# ---- the fused batch as a handle: fp_batch_create / permute / symbolic ----

def test_batch_handle_trio_matches_fused_order():
    """create + permute + symbolic on the union handle gives exactly what
    fp_batch_order gives; the perms are out after permute, the symbolic
    outputs after symbolic; with a network attached, the learned choices."""
    meshes = _mix(10, 41, 1500, 30000) + _tiny_meshes()
    caps = [128, 256, 384, 512, 200] * 2 + [16, 16, 4, 2, 40]
    ns = [m.n for m in meshes]
    faces = [torch.from_numpy(m.faces).cuda() for m in meshes]
    a = fp.make_batch(faces, ns, caps)
    b = fp.make_batch(faces, ns, caps)
    assert fp.fp_batch_order(a, fp.fp_default_options(), n_workers=0) == 0
    for _, outs in b.tensors:
        outs[2].fill_(-7)
    h = fp.fp_batch_create(b)
    try:
        fp.fp_batch_permute(h, b)
        torch.cuda.synchronize()
        for m, (_, ox), (_, oy) in zip(meshes, a.tensors, b.tensors):
            assert torch.equal(ox[0][:m.n], oy[0][:m.n]) and torch.equal(ox[1][:m.n], oy[1][:m.n])
            assert (oy[2] == -7).all()               # parents only after symbolic
        fp.fp_batch_symbolic(h, b)
        assert fp.fp_get_tree(h) >= 1                # the union's tree
        assert b[0].launches > 0
    finally:
        fp.fp_destroy(h)
    torch.cuda.synchronize()
    for m, x, y, (_, ox), (_, oy) in zip(meshes, a, b, a.tensors, b.tensors):
        assert (x.nnzL, x.flops, x.chosen_cap, x.status) == (y.nnzL, y.flops, y.chosen_cap, y.status)
        for tx, ty in zip(ox, oy):
            assert torch.equal(tx[:m.n], ty[:m.n])
    _check_item(meshes[3], b[3], b.tensors[3][1])
    # learned: the network attached to the union handle
    codes = fp.pack_params(M.gnn_weights(31), np.int32)
    c = fp.make_batch(faces, ns, caps)
    d = fp.make_batch(faces, ns, caps)
    assert fp.fp_batch_order_learned(c, codes, fp.fp_default_options(), n_workers=0) == 0
    h = fp.fp_batch_create(d)
    try:
        fp.fp_set_priority_net(h, codes)
        fp.fp_batch_permute(h, d)
        fp.fp_batch_symbolic(h, d)
    finally:
        fp.fp_destroy(h)
    torch.cuda.synchronize()
    for m, x, y, (_, ox), (_, oy) in zip(meshes, c, d, c.tensors, d.tensors):
        assert (x.nnzL, x.learned_leaves, x.learned_kept, x.fill_plain, x.fill_chosen) == \
            (y.nnzL, y.learned_leaves, y.learned_kept, y.fill_plain, y.fill_chosen)
        assert torch.equal(ox[0][:m.n], oy[0][:m.n])


def test_batch_handle_errors():
    meshes = _mix(3, 43)
    ns = [m.n for m in meshes]
    faces = [torch.from_numpy(m.faces).cuda() for m in meshes]
    items = fp.make_batch(faces, ns, [256] * 3)
    with pytest.raises(fp.FpError) as e:
        fp.fp_batch_create(items, fp.fp_default_options(dof_per_vertex=3))
    assert e.value.status == 1
    bad = torch.tensor([[0, 1, 12]], dtype=torch.int32, device="cuda")   # vertex 12 of a 10-vertex mesh
    with pytest.raises(fp.FpError) as e:
        fp.fp_batch_create(fp.make_batch(faces + [bad], ns + [10], [256] * 4))
    assert e.value.status == 1
    h = fp.fp_batch_create(items)
    try:
        with pytest.raises(fp.FpError) as e:
            fp.fp_batch_symbolic(h, items)                   # before permute
        assert e.value.status == 6
        assert fp.lib().fp_batch_permute(h, items, 2) == 1   # count differs from the create call
        fp.fp_batch_permute(h, items)
        fp.fp_batch_symbolic(h, items)
    finally:
        fp.fp_destroy(h)
    for m, it, (_, outs) in zip(meshes, items, items.tensors):
        _check_item(m, it, outs)
    single = fp.fp_create_from_faces(faces[0], ns[0], fp.fp_default_options())
    try:
        assert fp.lib().fp_batch_permute(single, items, 3) == 1   # not a batch handle
    finally:
        fp.fp_destroy(single)
