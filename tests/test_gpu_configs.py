"""Bit-exact parity with the oracle on every configuration at full size:
  - the 1024x1024 flipped torus with 3 DOF per vertex for seeds 1-4 (seed 0
    is in test_gpu_parity.py);
  - every one of the 256 meshes of the batch (n log-uniform in 2k-200k,
    grid / icosphere / flipped torus), each against the oracle run alone with
    the cap the autotuner chose for it;
  - the 2048x2048 flipped torus (4,194,304 vertices) of the learned batch,
    ordered with the GPU-trained network, against the oracle's learned
    ordering (the same network's codes, exact integer arithmetic).
The oracle runs in a process pool started with `spawn` before the first GPU
call of each test."""
import multiprocessing as mp
import os

import numpy as np
import pytest
import torch

import meshgen as M
import oracle_jobs as J

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _fp():
    import paper_2602_00898_b300 as fp
    return fp


def _pool(n):
    return mp.get_context("spawn").Pool(processes=max(1, min(n, os.cpu_count() or 1)), initializer=J.init_worker)


def _np(t):
    return t.cpu().numpy()


def test_torus1024_dof3_seeds_1_to_4():
    seeds = [1, 2, 3, 4]
    with _pool(len(seeds)) as pool:
        jobs = {s: pool.apply_async(J.torus_dof, (s,)) for s in seeds}
        fp = _fp()
        for s in seeds:
            mesh = M.torus1024(s)
            r = fp.order_faces(torch.from_numpy(mesh.faces).cuda(), mesh.n, patch_cap=512, dof_per_vertex=3)
            want = jobs[s].get()
            assert r.k == want["k"], s
            np.testing.assert_array_equal(_np(r.gmap), want["label"])
            np.testing.assert_array_equal(_np(r.node_of), want["node_of"])
            np.testing.assert_array_equal(_np(r.perm), want["perm"])
            np.testing.assert_array_equal(_np(r.parent), want["parent"])
            np.testing.assert_array_equal(_np(r.colcount), want["colcount"])
            assert r.nnzL == 9 * want["nnzL_vertex"] - 3 * want["n"]


def test_full_batch_256_every_mesh():
    """All 256 meshes of the batch workload, bit for bit."""
    meshes = M.mesh_mix(256, seed=0)
    with _pool(16) as pool:
        fp = _fp()
        faces = [torch.from_numpy(m.faces).cuda() for m in meshes]
        items = fp.make_batch(faces, [m.n for m in meshes])
        fp.fp_batch_autotune(items, fp.fp_default_options())
        st = fp.fp_batch_order(items, fp.fp_default_options())
        torch.cuda.synchronize()
        assert st == 0
        caps = [int(it.chosen_cap) for it in items]
        jobs = [pool.apply_async(J.mesh_plain, (m.faces, m.n, c)) for m, c in zip(meshes, caps)]
        for i, (m, it, (_, outs), job) in enumerate(zip(meshes, items, items.tensors, jobs)):
            want = job.get()
            perm, iperm, parent, colcount = [_np(t)[:m.n] for t in outs]
            np.testing.assert_array_equal(perm, want["perm"], err_msg=f"mesh {i}")
            np.testing.assert_array_equal(iperm[perm], np.arange(m.n))
            np.testing.assert_array_equal(parent, want["parent"], err_msg=f"mesh {i}")
            np.testing.assert_array_equal(colcount, want["colcount"], err_msg=f"mesh {i}")
            assert (it.nnzL, it.flops) == (want["nnzL"], want["flops"]), i


def test_learned_torus2048_matches_oracle():
    """The 4.2M-vertex torus of the learned batch with the trained network
    (cap 512): permutation, etree, column counts and the choice statistics."""
    from paper_2602_00898_b300.train_priorities import load_codes
    mesh = M.shuffle(M.torus(2048, 2048, 0.3, 4096), 4096)
    codes = np.asarray(load_codes(), np.int32)
    with _pool(1) as pool:
        job = pool.apply_async(J.mesh_learned, (mesh.faces, mesh.n, 512, codes))
        fp = _fp()
        faces = torch.from_numpy(mesh.faces).cuda()
        h = fp.fp_create_from_faces(faces, mesh.n, fp.fp_default_options(patch_cap=512))
        try:
            fp.fp_set_priority_net(h, codes)
            perm = torch.empty(mesh.n, dtype=torch.int32, device="cuda")
            fp.fp_permute(h, perm)
            parent = torch.empty_like(perm)
            colcount = torch.empty_like(perm)
            nnz, fl = fp.fp_symbolic(h, parent, colcount)
            leaves, kept, _, _ = fp.fp_learned_stats(h)
        finally:
            fp.fp_destroy(h)
        want = job.get(timeout=1800)
    np.testing.assert_array_equal(_np(perm), want["perm"])
    np.testing.assert_array_equal(_np(parent), want["parent"])
    np.testing.assert_array_equal(_np(colcount), want["colcount"])
    assert (nnz, fl) == (want["nnzL"], want["flops"])
    assert (leaves, kept) == (want["leaves"], want["kept"])
    assert nnz <= want["nnzL_plain"]
