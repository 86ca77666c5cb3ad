"""a10 training on the GPU against the oracle: samples (features, within-leaf
graph, best-of-nine ranks and targets) bit for bit, the float network's loss and
gradient within 1e-3 relative of the FP64 oracle, determinism of the step,
the SGD update and the quantisation, and what a trained network gains."""
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


def _sample(fp, mesh, cap, n_seeds=8):
    faces = torch.from_numpy(mesh.faces).cuda()
    h = fp.fp_create_from_faces(faces, mesh.n, fp.fp_default_options(patch_cap=cap))
    try:
        perm = torch.empty(mesh.n, dtype=torch.int32, device="cuda")
        fp.fp_permute(h, perm)
        s = fp.fp_gnn_sample(h, n_seeds)
        torch.cuda.synchronize()
        return s, perm.cpu().numpy()
    finally:
        fp.fp_destroy(h)


@pytest.mark.parametrize("seed,cap", [(0, 256), (2, 128)])
def test_sample_matches_oracle(seed, cap):
    fp = _fp()
    mesh = meshgen.grid64(seed)
    s, perm = _sample(fp, mesh, cap)
    g = O.graph_from_faces(mesh.faces, mesh.n)
    o = O.order(g, cap, seed=0)
    assert (perm == o.perm).all()
    lg = G.leaf_graph(g, o)
    X = G.features(g, o, cap, lg)
    T = G.targets(g, o, 8)
    x = s.x.cpu().numpy().reshape(-1, 8).astype(np.int64)
    assert (x[:, :6] == X).all()
    assert (s.mask.cpu().numpy().astype(bool) == lg.is_leaf).all()
    assert (s.lrowptr.cpu().numpy() == lg.rowptr).all()
    assert (s.lcol.cpu().numpy() == lg.col).all()
    assert (s.rank.cpu().numpy() == T.rank).all()
    np.testing.assert_allclose(s.target.cpu().numpy(), T.target, rtol=0, atol=1e-6)


def _float_params(seed):
    return {k: np.asarray(v, np.float64) for k, v in meshgen.gnn_weights(seed, quantized=False).items()}


def test_gradient_matches_oracle():
    fp = _fp()
    mesh = meshgen.grid64(1)
    s, _ = _sample(fp, mesh, 256)
    g = O.graph_from_faces(mesh.faces, mesh.n)
    o = O.order(g, 256)
    lg = G.leaf_graph(g, o)
    X = G.features(g, o, 256, lg) / 64.0
    T = G.targets(g, o, 8).target
    P = _float_params(4)
    loss_o, grad_o = G.loss_and_grad(P, X, lg, T)
    flat_o = fp.pack_params(grad_o, np.float64)
    params = torch.from_numpy(fp.pack_params(P, np.float32)).cuda()
    grad = torch.zeros_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    work = fp.gnn_work(s.n)
    fp.fp_gnn_train_step(params, grad, s, 0.0, loss, work)
    torch.cuda.synchronize()
    gg = grad.cpu().numpy().astype(np.float64)
    scale = np.abs(flat_o).max()
    assert abs(loss.item() - loss_o) <= 1e-4 * abs(loss_o)
    err = np.abs(gg - flat_o) / np.maximum(np.abs(flat_o), 1e-2 * scale)
    assert err.max() <= 1e-3, (err.argmax(), gg[err.argmax()], flat_o[err.argmax()])
    # lr = 0 leaves the parameters untouched
    assert (params.cpu().numpy() == fp.pack_params(P, np.float32)).all()


def test_step_is_deterministic_and_updates():
    fp = _fp()
    mesh = meshgen.shuffle(meshgen.torus(40, 30, 0.3, 2), 2)
    s, _ = _sample(fp, mesh, 128)
    P0 = fp.pack_params(_float_params(6), np.float32)
    outs = []
    for _ in range(2):
        params = torch.from_numpy(P0.copy()).cuda()
        grad = torch.zeros_like(params)
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        work = fp.gnn_work(s.n)
        fp.fp_gnn_train_step(params, grad, s, 0.01, loss, work)
        torch.cuda.synchronize()
        outs.append((params.cpu().numpy(), grad.cpu().numpy(), loss.item()))
    assert (outs[0][0] == outs[1][0]).all() and (outs[0][1] == outs[1][1]).all() and outs[0][2] == outs[1][2]
    np.testing.assert_allclose(outs[0][0], P0 - np.float32(0.01) * outs[0][1], rtol=0, atol=1e-7)
    # a few steps reduce the loss
    params = torch.from_numpy(P0.copy()).cuda()
    grad = torch.zeros_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    work = fp.gnn_work(s.n)
    losses = []
    for _ in range(8):
        fp.fp_gnn_train_step(params, grad, s, 0.02, loss, work)
        losses.append(loss.item())
    assert losses[-1] < losses[0]


def test_quantise_matches_oracle():
    fp = _fp()
    P = _float_params(9)
    params = torch.from_numpy(fp.pack_params(P, np.float32)).cuda()
    codes = torch.zeros(fp.GNN_NPARAMS, dtype=torch.int32, device="cuda")
    fp.fp_gnn_quantise(params, codes)
    torch.cuda.synchronize()
    q = G.quantise({k: np.asarray(v, np.float32).astype(np.float64) for k, v in P.items()})
    want = fp.pack_params({"w1s": q.w1s, "w1n": q.w1n, "b1": q.b1, "w2s": q.w2s, "w2n": q.w2n, "b2": q.b2,
                           "w3": q.w3, "c": q.c}, np.int32)
    assert (codes.cpu().numpy() == want).all()


def test_trained_network_gain_over_plain():
    """Train on a few meshes on the GPU, then order held-out meshes: the learned
    form never has more fill than plain minimum degree and, summed over the
    held-out set, has less."""
    fp = _fp()
    train = [meshgen.shuffle(meshgen.torus(30 + 4 * i, 28, 0.3, 100 + i), 100 + i) for i in range(6)]
    samples = [_sample(fp, m, 128)[0] for m in train]
    P = torch.from_numpy(fp.pack_params(_float_params(21), np.float32) * np.float32(0.5)).cuda()
    grad = torch.zeros_like(P)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    work = fp.gnn_work(max(s.n for s in samples))
    first = last = None
    for epoch in range(20):
        for s in samples:
            fp.fp_gnn_train_step(P, grad, s, 0.02, loss, work)
            if first is None:
                first = loss.item()
        last = loss.item()
    codes = torch.zeros(fp.GNN_NPARAMS, dtype=torch.int32, device="cuda")
    fp.fp_gnn_quantise(P, codes)
    codes = codes.cpu().numpy()
    gain, plain_total = 0, 0
    for i in range(4):
        m = meshgen.shuffle(meshgen.torus(36, 36, 0.3, 500 + i), 500 + i)
        f = torch.from_numpy(m.faces).cuda()
        a = fp.order_faces(f, m.n, patch_cap=128)
        b = fp.order_faces(f, m.n, patch_cap=128, net=codes)
        assert b.nnzL <= a.nnzL
        gain += a.nnzL - b.nnzL
        plain_total += a.nnzL
    print(f"training loss {first:.4f} -> {last:.4f}; held-out nnz(L) {plain_total} -> {plain_total - gain}")
    assert last < first
    assert gain > 0
