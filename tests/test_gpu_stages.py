"""Stage-by-stage parity: with debug_dump on, the library keeps every stage
boundary of Algorithm 1 (seeds, the labels after each Lloyd round, the
quotient graph, the side and the move of every patch at every dissection
level); each is compared element by element with the oracle's trace of the
same stage. Also the bounded device wait: a max_spin too small for the
tensor cores to finish makes the learned path fail with FP_ERR_TIMEOUT,
poisons the handle and leaves the device usable."""
import ctypes

import numpy as np
import pytest
import torch

import meshgen
import oracle as O

pytestmark = pytest.mark.gpu


def _fp():
    import paper_2602_00898_b300 as fp
    return fp


CASES = {
    "grid64_s0": lambda: (meshgen.grid64(0), 256, 0, 2),
    "grid64_s4": lambda: (meshgen.grid64(4), 64, 4, 2),
    "ico5": lambda: (meshgen.shuffle(meshgen.icosphere(5), 3), 128, 3, 3),
    "torus96": lambda: (meshgen.shuffle(meshgen.torus(96, 80, 0.3, 6), 6), 200, 6, 1),
    "disconnected": lambda: (_disconnected(), 40, 2, 2),
}


def _disconnected():
    """A torus, an icosphere and five isolated vertices in one mesh."""
    a = meshgen.shuffle(meshgen.torus(20, 14, 0.3, 1), 1)
    b = meshgen.shuffle(meshgen.icosphere(3), 4)
    f = np.concatenate([a.faces, b.faces + a.n]).astype(np.int32)
    return meshgen.Mesh("union", a.n + b.n + 5, f)


def _stage(fp, h, name, index=0):
    return fp.fp_get_stage(h, name, index).cpu().numpy()


@pytest.mark.parametrize("name", list(CASES))
def test_stages_match_oracle_trace(name):
    fp = _fp()
    mesh, cap, seed, rounds = CASES[name]()
    faces = torch.from_numpy(mesh.faces).cuda()
    opts = fp.fp_default_options(patch_cap=cap, seed=seed, lloyd_rounds=rounds, debug_dump=1)
    h = fp.fp_create_from_faces(faces, mesh.n, opts)
    try:
        perm = torch.empty(mesh.n, dtype=torch.int32, device="cuda")
        fp.fp_permute(h, perm)
        k = fp.fp_get_patches(h)
        depth = fp.fp_get_tree(h)
        got = {"seeds": _stage(fp, h, "seeds"),
               "labels": [_stage(fp, h, "labels", r) for r in range(rounds + 1)],
               "lloyd": [_stage(fp, h, "lloyd_seeds", r) for r in range(rounds)],
               "qw": _stage(fp, h, "quotient_weight"), "qr": _stage(fp, h, "quotient_rowptr"),
               "qc": _stage(fp, h, "quotient_col"), "qe": _stage(fp, h, "quotient_edge_weight")}
        levels = min(depth, int(np.ceil(np.log2(max(k, 1)))))
        got["side"] = [_stage(fp, h, "side", d) for d in range(levels)]
        got["child"] = [_stage(fp, h, "child", d) for d in range(levels)]
        torch.cuda.synchronize()
    finally:
        fp.fp_destroy(h)
    g = O.graph_from_faces(mesh.faces, mesh.n)
    t = O.order_trace(g, cap, seed=seed, lloyd_rounds=rounds)
    o = t.ordering
    assert (perm.cpu().numpy() == o.perm).all()
    assert k == o.k and depth == o.depth
    assert np.array_equal(got["seeds"], t.seeds0)
    for r in range(rounds + 1):
        assert np.array_equal(got["labels"][r], t.labels[r]), f"labels after round {r}"
    for r in range(rounds):
        assert np.array_equal(got["lloyd"][r], t.lloyd_seeds[r]), f"seeds after Lloyd round {r}"
    w, qr, qc, qe = O.quotient(g, o.label, o.k)
    assert np.array_equal(got["qw"], w)
    assert np.array_equal(got["qr"], qr)
    assert np.array_equal(got["qc"], qc)
    assert np.array_equal(got["qe"], qe)
    for d in range(levels):
        assert np.array_equal(got["side"][d], t.side_at[d]), f"sides at depth {d}"
        assert np.array_equal(got["child"][d], t.child_at[d]), f"moves at depth {d}"
    # the oracle bisects nothing below the recorded levels
    assert (t.side_at[levels:] == -1).all()


def test_stages_with_supplied_patches():
    """Sides and moves over caller-supplied groups (scattered, with an empty
    label) match the oracle's trace of the same groups."""
    fp = _fp()
    mesh = meshgen.shuffle(meshgen.grid(40, 30), 5)
    rng = np.random.default_rng(9)
    k = 23
    gmap = rng.integers(0, k, mesh.n).astype(np.int32)
    gmap[gmap == 7] = 8                      # label 7 stays empty
    faces = torch.from_numpy(mesh.faces).cuda()
    h = fp.fp_create_from_faces(faces, mesh.n, fp.fp_default_options(debug_dump=1))
    try:
        fp.fp_set_patches(h, torch.from_numpy(gmap).cuda(), k)
        perm = torch.empty(mesh.n, dtype=torch.int32, device="cuda")
        fp.fp_permute(h, perm)
        depth = fp.fp_get_tree(h)
        sides = [_stage(fp, h, "side", d) for d in range(depth)]
        child = [_stage(fp, h, "child", d) for d in range(depth)]
    finally:
        fp.fp_destroy(h)
    g = O.graph_from_faces(mesh.faces, mesh.n)
    t = O.order_trace(g, given=gmap, k=k)
    assert (perm.cpu().numpy() == t.ordering.perm).all()
    for d in range(depth):
        assert np.array_equal(sides[d], t.side_at[d]), d
        assert np.array_equal(child[d], t.child_at[d]), d


def test_stage_records_need_debug_dump():
    fp = _fp()
    mesh = meshgen.grid64(0)
    faces = torch.from_numpy(mesh.faces).cuda()
    h = fp.fp_create_from_faces(faces, mesh.n, fp.fp_default_options(patch_cap=256))
    try:
        fp.fp_permute(h)
        with pytest.raises(fp.FpError) as e:
            fp.fp_get_stage(h, "seeds")
        assert e.value.status == 6
    finally:
        fp.fp_destroy(h)
    h = fp.fp_create_from_faces(faces, mesh.n, fp.fp_default_options(patch_cap=256, debug_dump=1))
    try:
        fp.fp_permute(h)
        with pytest.raises(fp.FpError) as e:
            fp.fp_get_stage(h, "side", 99)            # no such level
        assert e.value.status == 6
        n = ctypes.c_int64()
        buf = torch.empty(4, dtype=torch.int32, device="cuda")
        st = fp.lib().fp_get_stage(h, 2, 0, buf.data_ptr(), 4, ctypes.byref(n))
        assert st == 1 and n.value == mesh.n          # buffer too small
    finally:
        fp.fp_destroy(h)


def test_bounded_wait_times_out_and_poisons_the_handle():
    """max_spin = 1: the scoring kernel gives up on its first poll of the
    tensor-core completion barrier, drains its MMA, frees its tensor memory
    and flags the failure; fp_permute returns FP_ERR_TIMEOUT, the handle
    answers FP_ERR_STATE afterwards, fp_destroy releases it, and the device
    keeps working (a fresh handle orders the same mesh bit-exactly)."""
    fp = _fp()
    mesh = meshgen.grid64(0)
    codes = fp.pack_params(meshgen.gnn_weights(3), np.int32)
    faces = torch.from_numpy(mesh.faces).cuda()
    L = fp.lib()
    h = fp.fp_create_from_faces(faces, mesh.n, fp.fp_default_options(patch_cap=256, max_spin=1))
    perm = torch.empty(mesh.n, dtype=torch.int32, device="cuda")
    try:
        fp.fp_set_priority_net(h, codes)
        st = L.fp_permute(h, perm.data_ptr(), None)
        assert st == 5, fp.fp_last_error(h)                     # FP_ERR_TIMEOUT
        assert "tensor-core" in fp.fp_last_error(h)
        assert L.fp_permute(h, perm.data_ptr(), None) == 6      # poisoned: FP_ERR_STATE
        nnz = ctypes.c_int64()
        assert L.fp_symbolic(h, None, None, ctypes.byref(nnz), None) == 6
    finally:
        assert L.fp_destroy(h) == 0
    torch.cuda.synchronize()
    # the same learned ordering with the default bound succeeds and matches
    # the oracle
    from oracle import gnn as G
    r = fp.order_faces(faces, mesh.n, patch_cap=256, net=codes)
    g = O.graph_from_faces(mesh.faces, mesh.n)
    o = O.order(g, 256)
    lo = G.order_learned(g, o, G.QParams.from_dict(meshgen.gnn_weights(3)), 256)
    assert (r.perm.cpu().numpy() == lo.perm).all()
