"""Parity of the learned priorities (a10) with the oracle: feature codes and
network scores element by element, the learned permutation, the per-leaf
choice statistics and nnz(L), all bit-exact (the network arithmetic is exact
integer arithmetic on the fixed-point grid)."""
import numpy as np
import pytest
import torch

import meshgen
import oracle as O
from oracle import gnn as G

pytestmark = pytest.mark.gpu


def _fp():
    import paper_2602_00898_b300 as fp
    return fp


MESHES = {
    "grid64_s0": lambda: (meshgen.grid64(0), 256),
    "grid64_s3": lambda: (meshgen.grid64(3), 256),
    "ico4": lambda: (meshgen.shuffle(meshgen.icosphere(4), 2), 128),
    "torus48": lambda: (meshgen.shuffle(meshgen.torus(48, 40, 0.3, 5), 5), 200),
    "grid7x5": lambda: (meshgen.shuffle(meshgen.grid(7, 5), 1), 16),
}


def _plain(fp, mesh, cap):
    faces = torch.from_numpy(mesh.faces).cuda()
    h = fp.fp_create_from_faces(faces, mesh.n, fp.fp_default_options(patch_cap=cap))
    return h, faces


@pytest.mark.parametrize("name", list(MESHES))
def test_features_and_scores_match_oracle(name):
    fp = _fp()
    mesh, cap = MESHES[name]()
    d = meshgen.gnn_weights(7)
    codes = fp.pack_params(d, np.int32)
    h, faces = _plain(fp, mesh, cap)
    try:
        perm = torch.empty(mesh.n, dtype=torch.int32, device="cuda")
        fp.fp_permute(h, perm)
        S = torch.zeros(mesh.n, dtype=torch.int32, device="cuda")
        X = torch.zeros(mesh.n * 8, dtype=torch.uint8, device="cuda")
        fp.fp_gnn_scores(h, codes, S, X)
        torch.cuda.synchronize()
    finally:
        fp.fp_destroy(h)
    g = O.graph_from_faces(mesh.faces, mesh.n)
    o = O.order(g, cap)
    assert (perm.cpu().numpy() == o.perm).all()
    lg = G.leaf_graph(g, o)
    Xo = G.features(g, o, cap, lg)
    So = G.forward_q(G.QParams.from_dict(d), Xo, lg)
    Xg = X.cpu().numpy().reshape(-1, 8).astype(np.int64)
    assert (Xg[:, :6] == Xo).all()
    assert (Xg[:, 6:] == 0).all()
    assert (S.cpu().numpy().astype(np.int64) == So).all()


@pytest.mark.parametrize("name,wseed", [("grid64_s0", 11), ("grid64_s3", 12), ("ico4", 13), ("torus48", 14),
                                        ("grid7x5", 15)])
def test_learned_order_matches_oracle(name, wseed):
    fp = _fp()
    mesh, cap = MESHES[name]()
    d = meshgen.gnn_weights(wseed)
    codes = fp.pack_params(d, np.int32)
    faces = torch.from_numpy(mesh.faces).cuda()
    h = fp.fp_create_from_faces(faces, mesh.n, fp.fp_default_options(patch_cap=cap))
    try:
        fp.fp_set_priority_net(h, codes)
        perm = torch.empty(mesh.n, dtype=torch.int32, device="cuda")
        iperm = torch.empty(mesh.n, dtype=torch.int32, device="cuda")
        fp.fp_permute(h, perm, iperm)
        parent = torch.empty(mesh.n, dtype=torch.int32, device="cuda")
        cc = torch.empty(mesh.n, dtype=torch.int32, device="cuda")
        nnz, fl = fp.fp_symbolic(h, parent, cc)
        leaves, kept, f_plain, f_chosen = fp.fp_learned_stats(h)
        torch.cuda.synchronize()
    finally:
        fp.fp_destroy(h)
    g = O.graph_from_faces(mesh.faces, mesh.n)
    o = O.order(g, cap)
    L = G.order_learned(g, o, G.QParams.from_dict(d), cap)
    p = perm.cpu().numpy()
    assert (p == L.perm).all()
    assert (iperm.cpu().numpy() == L.iperm).all()
    assert leaves == len(L.leaves) and kept == int(L.kept.sum())
    assert f_plain == int(L.fill_plain.sum())
    assert f_chosen == int(np.where(L.kept, L.fill_learned, L.fill_plain).sum())
    sym = O.symbolic(g, L.perm)
    assert nnz == sym.nnzL and fl == sym.flops
    assert (parent.cpu().numpy() == sym.parent).all() and (cc.cpu().numpy() == sym.colcount).all()
    assert nnz <= O.symbolic(g, o.perm).nnzL


def test_constant_network_keeps_plain_orders():
    fp = _fp()
    mesh, cap = MESHES["grid64_s0"]()
    d = {k: np.zeros_like(np.asarray(v)) for k, v in meshgen.gnn_weights(0).items()}
    res = fp.order_faces(torch.from_numpy(mesh.faces).cuda(), mesh.n, patch_cap=cap, net=fp.pack_params(d, np.int32))
    plain = fp.order_faces(torch.from_numpy(mesh.faces).cuda(), mesh.n, patch_cap=cap)
    assert (res.perm.cpu() == plain.perm.cpu()).all() and res.nnzL == plain.nnzL


def test_bad_codes_rejected():
    fp = _fp()
    mesh, cap = MESHES["grid7x5"]()
    faces = torch.from_numpy(mesh.faces).cuda()
    h = fp.fp_create_from_faces(faces, mesh.n, fp.fp_default_options(patch_cap=cap))
    try:
        codes = np.zeros(fp.GNN_NPARAMS, np.int32)
        codes[0] = 256                      # weight code beyond 255
        with pytest.raises(fp.FpError):
            fp.fp_set_priority_net(h, codes)
    finally:
        fp.fp_destroy(h)


def test_learned_full_size_properties():
    """1M-vertex flipped torus with the GPU-trained network: properties that
    hold for any network. Every leaf keeps its vertex set and position range,
    separators do not move, the permutation is a bijection, and nnz(L) is at
    most the plain method's, lower by exactly the kept leaves' fill gains."""
    fp = _fp()
    from paper_2602_00898_b300.train_priorities import load_codes
    mesh = meshgen.torus1024()
    faces = torch.from_numpy(mesh.faces).cuda()
    plain = fp.order_faces(faces, mesh.n, patch_cap=512)
    h = fp.fp_create_from_faces(faces, mesh.n, fp.fp_default_options(patch_cap=512))
    try:
        fp.fp_set_priority_net(h, load_codes())
        perm = torch.empty(mesh.n, dtype=torch.int32, device="cuda")
        fp.fp_permute(h, perm)
        nnz, _ = fp.fp_symbolic(h)
        leaves, kept, f_plain, f_chosen = fp.fp_learned_stats(h)
    finally:
        fp.fp_destroy(h)
    p_l = perm.cpu().numpy()
    p_p = plain.perm.cpu().numpy()
    assert np.array_equal(np.sort(p_l), np.arange(mesh.n))
    nb = plain.node_begin.cpu().numpy()
    ns = plain.node_size.cpu().numpy()
    sub = ns.astype(np.int64).copy()
    for t in range(ns.size - 1, -1, -1):
        for c in (2 * t + 1, 2 * t + 2):
            if c < ns.size:
                sub[t] += sub[c]
    is_leaf_pos = np.zeros(mesh.n, bool)
    nleaves = 0
    for t in range(ns.size):
        if 0 < ns[t] <= 512 and sub[t] == ns[t]:
            nleaves += 1
            a, b = nb[t], nb[t] + ns[t]
            is_leaf_pos[a:b] = True
            assert np.array_equal(np.sort(p_l[a:b]), np.sort(p_p[a:b]))
    assert leaves == nleaves and kept > 0
    assert np.array_equal(p_l[~is_leaf_pos], p_p[~is_leaf_pos])
    assert nnz <= plain.nnzL and plain.nnzL - nnz == f_plain - f_chosen
