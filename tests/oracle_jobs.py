"""Oracle runs for the full-size parity tests, as plain functions that a
process pool started with `spawn` can import. Test infrastructure only: each
job calls the CPU oracle on one input and returns its results."""
from __future__ import annotations

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def init_worker():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)


def torus_dof(seed: int, cap: int = 512, dof: int = 3):
    """The 1024x1024 flipped torus of `seed`: ordering, symbolic factor and
    their DOF expansion."""
    import meshgen as M
    import oracle as O
    mesh = M.torus1024(seed)
    g = O.graph_from_faces(mesh.faces, mesh.n)
    o = O.order(g, cap, seed=0)
    s = O.symbolic(g, o.perm)
    pd, ad, cd = O.dof_expand(dof, o.perm, s.parent, s.colcount)
    return {"n": g.n, "perm": pd, "parent": ad, "colcount": cd, "nnzL_vertex": s.nnzL, "label": o.label,
            "node_of": o.node_of, "k": o.k}


def mesh_plain(faces, n: int, cap: int):
    """Ordering and symbolic factor of one mesh alone."""
    import oracle as O
    g = O.graph_from_faces(faces, n)
    o = O.order(g, cap, seed=0)
    s = O.symbolic(g, o.perm)
    return {"perm": o.perm, "parent": s.parent, "colcount": s.colcount, "nnzL": s.nnzL, "flops": s.flops}


def mesh_learned(faces, n: int, cap: int, codes):
    """The learned ordering (plain ordering, then the network's leaf choices)
    and its symbolic factor."""
    import paper_2602_00898_b300 as fp
    import oracle as O
    from oracle import gnn as G
    g = O.graph_from_faces(faces, n)
    o = O.order(g, cap, seed=0)
    L = G.order_learned(g, o, G.QParams.from_dict(fp.unpack_params(codes)), cap)
    s = O.symbolic(g, L.perm)
    plain = O.symbolic(g, o.perm)
    return {"perm": L.perm, "parent": s.parent, "colcount": s.colcount, "nnzL": s.nnzL, "flops": s.flops,
            "nnzL_plain": plain.nnzL, "leaves": len(L.leaves), "kept": int(L.kept.sum())}
