"""Trains the leaf-priority network of the learned orderings on the GPU.

Training set: `--meshes` synthetic meshes (default 2,000) of 2k-50k vertices
(grid, icosphere and flipped-torus types mixed by seed, shuffled ids), from a
seed stream disjoint from the evaluation meshes. For each mesh the library
computes the plain ordering and a training sample (fp_gnn_sample: feature
codes, within-leaf graph, and as targets the normalised ranks of the lowest-
fill order among plain minimum degree and eight seeded minimum-degree orders),
then runs `--epochs` passes of full-sample gradient steps (fp_gnn_train_step,
one mesh per step, fixed order) and quantises the weights (fp_gnn_quantise).
The codes and a summary (training losses, held-out nnz(L) against the plain
method) are written as JSON, by default next to this file as
priority_net.json, which the batched learned benchmark loads.

    python -m paper_2602_00898_b300.train_priorities [--meshes 2000] [--epochs 3]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "priority_net.json")
TRAIN_SEED = 1_000_003      # mesh_mix seed of the training set
HOLDOUT_SEED = 2_000_003    # mesh_mix seed of the held-out check
INIT_SEED = 21              # seeded initial float weights


def load_codes(path: str = DEFAULT_OUT) -> np.ndarray:
    """The trained codes (int32 [FP_GNN_NPARAMS]) from a file this script wrote."""
    with open(path) as f:
        return np.asarray(json.load(f)["codes"], dtype=np.int32)


def main(argv=None) -> dict:
    import torch

    import meshgen
    from . import (fp_create_from_faces, fp_default_options, fp_destroy, fp_gnn_quantise, fp_gnn_sample,
                   fp_gnn_train_step, fp_permute, gnn_work, order_faces, pack_params, GNN_NPARAMS)

    ap = argparse.ArgumentParser()
    ap.add_argument("--meshes", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--lr", type=float, default=0.02)
    ap.add_argument("--cap", type=int, default=512)
    ap.add_argument("--holdout", type=int, default=32)
    ap.add_argument("--out", default=DEFAULT_OUT)
    args = ap.parse_args(argv)

    t0 = time.time()
    meshes = meshgen.mesh_mix(args.meshes, TRAIN_SEED, 2000, 50000)
    samples = []
    for m in meshes:
        faces = torch.from_numpy(m.faces).cuda()
        h = fp_create_from_faces(faces, m.n, fp_default_options(patch_cap=args.cap))
        try:
            fp_permute(h)
            samples.append(fp_gnn_sample(h, 8))
        finally:
            fp_destroy(h)
    torch.cuda.synchronize()
    t_samples = time.time() - t0

    w = meshgen.gnn_weights(INIT_SEED, quantized=False)
    P = torch.from_numpy(pack_params(w, np.float32) * np.float32(0.5)).cuda()
    grad = torch.zeros_like(P)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    work = gnn_work(max(s.n for s in samples))
    epoch_loss = []
    for _ in range(args.epochs):
        acc = torch.zeros(1, dtype=torch.float64, device="cuda")
        for s in samples:
            fp_gnn_train_step(P, grad, s, args.lr, loss, work)
            acc += loss.double()
        epoch_loss.append(float(acc.item() / len(samples)))
    codes = torch.zeros(GNN_NPARAMS, dtype=torch.int32, device="cuda")
    fp_gnn_quantise(P, codes)
    torch.cuda.synchronize()
    codes = codes.cpu().numpy()
    t_train = time.time() - t0 - t_samples

    plain = learned = 0
    for m in meshgen.mesh_mix(args.holdout, HOLDOUT_SEED, 2000, 50000):
        f = torch.from_numpy(m.faces).cuda()
        plain += order_faces(f, m.n, patch_cap=args.cap).nnzL
        learned += order_faces(f, m.n, patch_cap=args.cap, net=codes).nnzL
    summary = {
        "codes": codes.tolist(),
        "training_meshes": args.meshes, "vertices": int(sum(m.n for m in meshes)), "epochs": args.epochs,
        "lr": args.lr, "patch_cap": args.cap, "init_seed": INIT_SEED, "train_seed": TRAIN_SEED,
        "epoch_loss": epoch_loss, "sample_seconds": round(t_samples, 1), "train_seconds": round(t_train, 1),
        "holdout": {"meshes": args.holdout, "seed": HOLDOUT_SEED, "nnzL_plain": int(plain),
                    "nnzL_learned": int(learned)},
    }
    with open(args.out, "w") as f:
        json.dump(summary, f)
    print(json.dumps({k: v for k, v in summary.items() if k != "codes"}))
    return summary


if __name__ == "__main__":
    main()
