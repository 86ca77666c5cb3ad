"""Seeded synthetic triangle meshes: the inputs shared by the tests, the
benchmark and the smoke check.

This module holds no step of the ordering method. It only produces face lists
(int32 [F, 3], vertex ids 0..n-1) whose connectivity matches the workload
families the paper evaluates on (scanned surface meshes, Section 6): regular
grid discs, icospheres and flipped tori, with vertex ids shuffled by seed so
that no ordering information leaks from the generator into the method.

Every function is deterministic in its arguments (numpy PCG64 streams).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Mesh:
    name: str
    n: int                 # number of vertices
    faces: np.ndarray      # int32 [F, 3]

    @property
    def n_faces(self) -> int:
        return int(self.faces.shape[0])


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed) & 0xFFFFFFFF, int(stream)]))


def shuffle(mesh: Mesh, seed: int) -> Mesh:
    """Relabel the vertices by a seeded random permutation."""
    pi = _rng(seed, 1).permutation(mesh.n).astype(np.int32)
    return Mesh(mesh.name, mesh.n, pi[mesh.faces].astype(np.int32))


def grid(nx: int, ny: int) -> Mesh:
    """nx*ny vertex grid; quad (i, j) -> (v00, v10, v11), (v00, v11, v01):
    every diagonal runs the same way."""
    i, j = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), indexing="ij")
    i = i.ravel(); j = j.ravel()
    v00 = i * ny + j
    v10 = (i + 1) * ny + j
    v01 = i * ny + j + 1
    v11 = (i + 1) * ny + j + 1
    f = np.concatenate([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)])
    return Mesh(f"grid{nx}x{ny}", nx * ny, f.astype(np.int32))


def torus(nx: int, ny: int, flip_p: float = 0.0, seed: int = 0) -> Mesh:
    """Periodic nx*ny torus grid; each quad's diagonal is flipped with
    probability flip_p (seeded)."""
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    i = i.ravel(); j = j.ravel()
    ip = (i + 1) % nx
    jp = (j + 1) % ny
    v00 = i * ny + j
    v10 = ip * ny + j
    v01 = i * ny + jp
    v11 = ip * ny + jp
    flip = _rng(seed, 2).random(nx * ny) < flip_p
    a = np.where(flip[:, None], np.stack([v00, v10, v01], 1), np.stack([v00, v10, v11], 1))
    b = np.where(flip[:, None], np.stack([v10, v11, v01], 1), np.stack([v00, v11, v01], 1))
    f = np.concatenate([a, b])
    return Mesh(f"torus{nx}x{ny}", nx * ny, f.astype(np.int32))


def icosphere(level: int) -> Mesh:
    """Icosahedron midpoint-subdivided `level` times: 10*4^level + 2 vertices.
    Vertex positions do not affect the matrix pattern, so only the
    connectivity is produced."""
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    n = 12
    for _ in range(level):
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
        lo = e.min(1); hi = e.max(1)
        key = lo * (n + 1) + hi
        uk, inv = np.unique(key, return_inverse=True)
        mid = n + inv.reshape(3, -1)          # midpoint ids of edges ab, bc, ca
        n = n + uk.size
        a, b, c = f[:, 0], f[:, 1], f[:, 2]
        ab, bc, ca = mid[0], mid[1], mid[2]
        f = np.concatenate([np.stack([a, ab, ca], 1), np.stack([b, bc, ab], 1),
                            np.stack([c, ca, bc], 1), np.stack([ab, bc, ca], 1)])
    return Mesh(f"icosphere{level}", n, f.astype(np.int32))


# --- named workloads --------------------------------------------------------

def grid64(seed: int = 0) -> Mesh:
    """64x64 grid (4,096 vertices), shuffled; patch cap 256."""
    return shuffle(grid(64, 64), seed)


def icosphere7(seed: int = 0) -> Mesh:
    """Icosphere level 7 (163,842 vertices, 327,680 faces), shuffled; cap 512."""
    return shuffle(icosphere(7), seed)


def torus1024(seed: int = 0, flip_p: float = 0.3) -> Mesh:
    """1024x1024 torus with 30% of diagonals flipped, shuffled (1,048,576 vertices)."""
    return shuffle(torus(1024, 1024, flip_p, seed), seed)


def mesh_mix(count: int, seed: int, n_lo: int = 2000, n_hi: int = 200000) -> list[Mesh]:
    """`count` meshes with vertex counts log-uniform in [n_lo, n_hi], type
    uniform over {grid, icosphere, flipped torus}, each shuffled by its own
    seed. Icospheres take the subdivision level whose size is nearest."""
    rng = _rng(seed, 3)
    out = []
    for m in range(count):
        target = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        kind = int(rng.integers(0, 3))
        s = int(rng.integers(0, 2**31 - 1))
        if kind == 0:
            side = max(2, int(round(math.sqrt(target))))
            msh = grid(side, side)
        elif kind == 1:
            lvl = min(range(2, 8), key=lambda L: abs((10 * 4**L + 2) - target))
            msh = icosphere(lvl)
        else:
            side = max(3, int(round(math.sqrt(target))))
            msh = torus(side, side, 0.3, s)
        out.append(shuffle(msh, s))
    return out


def gnn_weights(seed: int, f_in: int = 6, hidden: int = 32, quantized: bool = True) -> dict:
    """Seeded random weights for the two-layer message-passing priority network
    (input width f_in, hidden width `hidden`, scalar head). quantized: integer
    codes (weights in [-48, 48], biases in [-4096, 4096], head bias in
    [-8192, 8192]); otherwise float64 values (weights ~ N(0, 0.25^2), biases
    ~ N(0, 0.1^2)). Only random numbers: the meaning of the codes belongs to
    the method."""
    r = _rng(seed, 7)
    shapes = {"w1s": (hidden, f_in), "w1n": (hidden, f_in), "b1": (hidden,), "w2s": (hidden, hidden),
              "w2n": (hidden, hidden), "b2": (hidden,), "w3": (hidden,), "c": ()}
    out = {}
    for k, sh in shapes.items():
        if quantized:
            lim = 8192 if k == "c" else (4096 if k.startswith("b") else 48)
            out[k] = r.integers(-lim, lim + 1, size=sh, dtype=np.int64)
        else:
            sd = 0.1 if k in ("b1", "b2", "c") else 0.25
            out[k] = r.normal(0.0, sd, size=sh)
    return out


def laplacian_values(rowptr: np.ndarray, col: np.ndarray, seed: int | None = None, shift: float = 1.0):
    """FP64 values of a graph Laplacian plus `shift` times the identity on the
    symmetric CSR pattern (rowptr, col): A_ij = -w_ij off the diagonal and
    A_ii = sum_j w_ij + shift. seed None: unit weights (the configurations'
    "Laplacian + I"); else symmetric weights uniform in [0.5, 1.5] drawn per
    undirected edge from a PCG64 stream. Returns (diag [n], off [nnz])."""
    n = rowptr.size - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    dst = col.astype(np.int64)
    if seed is None:
        w = np.ones(dst.size)
    else:
        key = np.minimum(src, dst) * n + np.maximum(src, dst)
        uk, inv = np.unique(key, return_inverse=True)
        w = _rng(seed, 7).uniform(0.5, 1.5, uk.size)[inv]
    diag = np.bincount(src, weights=w, minlength=n) + shift
    return diag, -w
