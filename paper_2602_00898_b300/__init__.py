"""Python binding of the fastperm C ABI (include/fastperm.h).

Argument marshalling only: every function forwards to the function of the same
name in libfastperm.so; PyTorch provides device memory and the CUDA stream.
There is no fallback: if the shared library cannot be loaded (or built with
nvcc), importing the binding's entry points raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from . import _build

_HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(_HERE), "include", "fastperm.h")

FP_OK = 0
STATUS = {0: "FP_OK", 1: "FP_ERR_INVALID_ARG", 2: "FP_ERR_NOT_SYMMETRIC", 3: "FP_ERR_OUT_OF_MEMORY",
          4: "FP_ERR_CUDA", 5: "FP_ERR_TIMEOUT", 6: "FP_ERR_STATE", 7: "FP_ERR_UNSUPPORTED"}


class FpError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class fp_options(ctypes.Structure):
    _fields_ = [("patch_cap", ctypes.c_int32), ("lloyd_rounds", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("nd_level", ctypes.c_int32), ("schedule", ctypes.c_int32), ("dof_per_vertex", ctypes.c_int32),
                ("debug_dump", ctypes.c_int32), ("max_spin", ctypes.c_int64)]


class fp_batch_item(ctypes.Structure):
    _fields_ = [("d_faces", ctypes.c_void_p), ("n_faces", ctypes.c_int64), ("n_vertices", ctypes.c_int32),
                ("patch_cap", ctypes.c_int32), ("d_perm", ctypes.c_void_p), ("d_iperm", ctypes.c_void_p),
                ("d_parent", ctypes.c_void_p), ("d_colcount", ctypes.c_void_p), ("nnzL", ctypes.c_int64),
                ("flops", ctypes.c_int64), ("chosen_cap", ctypes.c_int32), ("status", ctypes.c_int32),
                ("launches", ctypes.c_int64), ("learned_leaves", ctypes.c_int32), ("learned_kept", ctypes.c_int32),
                ("fill_plain", ctypes.c_int64), ("fill_chosen", ctypes.c_int64)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load (building in-tree if stale) libfastperm.so."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        P32, P64 = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
        opt = ctypes.POINTER(fp_options)
        sig = {
            "fp_default_options": (None, [opt]),
            "fp_create_from_faces": (i32, [vp, i64, i32, opt, vp, ctypes.POINTER(vp)]),
            "fp_create_from_csr": (i32, [vp, vp, i32, opt, vp, ctypes.POINTER(vp)]),
            "fp_permute": (i32, [vp, vp, vp]),
            "fp_symbolic": (i32, [vp, vp, vp, P64, P64]),
            "fp_get_sizes": (i32, [vp, P32, P32, P64]),
            "fp_get_stage": (i32, [vp, i32, i32, vp, i64, P64]),
            "fp_factor": (i32, [vp, vp, vp]),
            "fp_solve": (i32, [vp, vp, vp]),
            "fp_factor_export": (i32, [vp, vp, vp, vp, i64, P64]),
            "fp_factor_stats": (i32, [vp, P64, P64, P64]),
            "fp_get_graph": (i32, [vp, vp, vp]),
            "fp_get_patches": (i32, [vp, vp, P32]),
            "fp_set_patches": (i32, [vp, vp, i32]),
            "fp_get_tree": (i32, [vp, P32, vp, vp, vp]),
            "fp_order_faces_host": (i32, [vp, i64, i32, opt, vp, vp, vp, vp, vp, P64, P64]),
            "fp_destroy": (i32, [vp]),
            "fp_last_error": (ctypes.c_char_p, [vp]),
            "fp_status_string": (ctypes.c_char_p, [i32]),
            "fp_launch_count": (i64, [vp]),
            "fp_profiling": (None, [ctypes.c_int]),
            "fp_profile_read": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), P64, ctypes.c_int]),
            "fp_profile_reset": (None, []),
            "fp_batch_order": (i32, [ctypes.POINTER(fp_batch_item), i32, opt, i32]),
            "fp_batch_autotune": (i32, [ctypes.POINTER(fp_batch_item), i32, opt, P32]),
            "fp_batch_order_learned": (i32, [ctypes.POINTER(fp_batch_item), i32, opt, i32, P32]),
            "fp_batch_create": (i32, [ctypes.POINTER(fp_batch_item), i32, opt, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_void_p)]),
            "fp_batch_permute": (i32, [ctypes.c_void_p, ctypes.POINTER(fp_batch_item), i32]),
            "fp_batch_symbolic": (i32, [ctypes.c_void_p, ctypes.POINTER(fp_batch_item), i32]),
            "fp_graph_from_faces_static": (i32, [vp, i64, i32, vp, vp, i64, P64, vp]),
            "fp_set_priority_net": (i32, [vp, P32]),
            "fp_learned_stats": (i32, [vp, P32, P32, P64, P64]),
            "fp_gnn_scores": (i32, [vp, P32, vp, vp]),
            "fp_gnn_sample": (i32, [vp, i32, vp, vp, vp, vp, vp, vp, i64, P64]),
            "fp_gnn_train_work_bytes": (i64, [i32]),
            "fp_gnn_train_step": (i32, [vp, vp, vp, vp, vp, vp, vp, i32, ctypes.c_float, vp, vp, i64, vp]),
            "fp_gnn_quantise": (i32, [vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(t) -> int | None:
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(stream)


def _check(status: int, h=None):
    if status != FP_OK:
        raise FpError(status, lib().fp_last_error(h).decode())


def fp_default_options(**kw) -> fp_options:
    o = fp_options()
    lib().fp_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def fp_create_from_faces(faces, n_vertices: int, opts: fp_options | None = None, stream=None):
    """faces: int32 CUDA tensor [F, 3]. Returns an opaque handle (c_void_p)."""
    opts = opts or fp_default_options()
    h = ctypes.c_void_p()
    nf = int(faces.shape[0]) if faces is not None else 0
    _check(lib().fp_create_from_faces(_ptr(faces) if nf else None, nf, int(n_vertices), ctypes.byref(opts),
                                      _stream(stream), ctypes.byref(h)))
    return h


def fp_create_from_csr(rowptr, col, n_rows: int, opts: fp_options | None = None, stream=None):
    opts = opts or fp_default_options()
    h = ctypes.c_void_p()
    _check(lib().fp_create_from_csr(_ptr(rowptr), _ptr(col) if col is not None and col.numel() else None,
                                    int(n_rows), ctypes.byref(opts), _stream(stream), ctypes.byref(h)))
    return h


def fp_permute(h, perm=None, iperm=None):
    _check(lib().fp_permute(h, _ptr(perm), _ptr(iperm)), h)


def fp_symbolic(h, parent=None, colcount=None) -> tuple[int, int]:
    nnz, fl = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().fp_symbolic(h, _ptr(parent), _ptr(colcount), ctypes.byref(nnz), ctypes.byref(fl)), h)
    return nnz.value, fl.value


def fp_get_sizes(h) -> tuple[int, int, int]:
    n, b, nnz = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(lib().fp_get_sizes(h, ctypes.byref(n), ctypes.byref(b), ctypes.byref(nnz)), h)
    return n.value, b.value, nnz.value


STAGES = {"seeds": 0, "lloyd_seeds": 1, "labels": 2, "quotient_weight": 3, "quotient_rowptr": 4,
          "quotient_col": 5, "quotient_edge_weight": 6, "side": 7, "child": 8}


def fp_get_stage(h, stage: str, index: int = 0):
    """A stage boundary of the last fp_permute of a handle created with
    debug_dump=1, as a new int32 CUDA tensor."""
    import torch
    n = ctypes.c_int64()
    code = STAGES[stage]
    _check(lib().fp_get_stage(h, code, int(index), None, 0, ctypes.byref(n)), h)
    out = torch.empty(max(n.value, 1), dtype=torch.int32, device="cuda")
    _check(lib().fp_get_stage(h, code, int(index), out.data_ptr(), n.value, ctypes.byref(n)), h)
    return out[:n.value]


def fp_factor(h, diag, offdiag):
    """Numeric Cholesky of P A P^T (A: FP64 CUDA tensors, diag [n] by vertex,
    offdiag [nnz] aligned with fp_get_graph's CSR)."""
    _check(lib().fp_factor(h, _ptr(diag), _ptr(offdiag)), h)


def fp_solve(h, b, x=None):
    """x with A x = b (FP64 CUDA tensors by vertex); returns x."""
    import torch
    if x is None:
        x = torch.empty_like(b)
    _check(lib().fp_solve(h, _ptr(b), _ptr(x)), h)
    return x


def fp_factor_export(h):
    """The factor as (colptr int64, rows int32, vals float64) CUDA tensors."""
    import torch
    nnz = ctypes.c_int64()
    _check(lib().fp_factor_export(h, None, None, None, 0, ctypes.byref(nnz)), h)
    n, _, _ = fp_get_sizes(h)
    dev = torch.device("cuda", torch.cuda.current_device())
    cp = torch.empty(n + 1, dtype=torch.int64, device=dev)
    ri = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=dev)
    rx = torch.empty(max(nnz.value, 1), dtype=torch.float64, device=dev)
    _check(lib().fp_factor_export(h, _ptr(cp), _ptr(ri), _ptr(rx), nnz.value, ctypes.byref(nnz)), h)
    return cp, ri[:nnz.value], rx[:nnz.value]


def fp_factor_stats(h) -> tuple[int, int, int]:
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().fp_factor_stats(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), h)
    return a.value, b.value, c.value


def fp_get_graph(h, rowptr=None, col=None):
    _check(lib().fp_get_graph(h, _ptr(rowptr), _ptr(col)), h)


def fp_get_patches(h, gmap=None) -> int:
    k = ctypes.c_int32()
    _check(lib().fp_get_patches(h, _ptr(gmap), ctypes.byref(k)), h)
    return k.value


def fp_set_patches(h, gmap, k: int):
    """Supplies the patch of every vertex (int32 CUDA tensor, values in [0, k));
    later fp_permute calls dissect over these groups instead of patching."""
    _check(lib().fp_set_patches(h, _ptr(gmap), int(k)), h)


def fp_get_tree(h, node_begin=None, node_size=None, node_of=None) -> int:
    d = ctypes.c_int32()
    _check(lib().fp_get_tree(h, ctypes.byref(d), _ptr(node_begin), _ptr(node_size), _ptr(node_of)), h)
    return d.value


def fp_order_faces_host(faces, n_vertices: int, opts: fp_options | None = None, stream=None,
                        perm=None, iperm=None, parent=None, colcount=None) -> tuple[int, int]:
    """Host-buffer form: faces and outputs are CPU tensors (pinned for speed)."""
    opts = opts or fp_default_options()
    nnz, fl = ctypes.c_int64(), ctypes.c_int64()
    nf = int(faces.shape[0])
    _check(lib().fp_order_faces_host(_ptr(faces) if nf else None, nf, int(n_vertices), ctypes.byref(opts),
                                     _stream(stream), _ptr(perm), _ptr(iperm), _ptr(parent), _ptr(colcount),
                                     ctypes.byref(nnz), ctypes.byref(fl)))
    return nnz.value, fl.value


def fp_destroy(h):
    if h:
        lib().fp_destroy(h)


def fp_last_error(h=None) -> str:
    return lib().fp_last_error(h).decode()


def fp_launch_count(h) -> int:
    return int(lib().fp_launch_count(h))


def fp_batch_order(items, opts: fp_options | None = None, n_workers: int = 0) -> int:
    """items: a ctypes array of fp_batch_item (filled in place). Returns the
    batch status; each item carries its own status, nnzL, flops, chosen_cap."""
    opts = opts or fp_default_options()
    return int(lib().fp_batch_order(items, len(items), ctypes.byref(opts), n_workers))


def fp_batch_order_learned(items, codes, opts: fp_options | None = None, n_workers: int = 0) -> int:
    """fp_batch_order with the priority network `codes` attached to every mesh."""
    import numpy as np
    opts = opts or fp_default_options()
    c = np.ascontiguousarray(codes, dtype=np.int32)
    assert c.size == GNN_NPARAMS
    return int(lib().fp_batch_order_learned(items, len(items), ctypes.byref(opts), n_workers,
                                            c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))


def fp_batch_create(items, opts: fp_options | None = None, stream=None):
    """The fused batch as one handle over the disjoint union of the items'
    meshes (items: a ctypes array of fp_batch_item). Returns the handle."""
    opts = opts or fp_default_options()
    h = ctypes.c_void_p()
    _check(lib().fp_batch_create(items, len(items), ctypes.byref(opts), _stream(stream), ctypes.byref(h)))
    return h


def fp_batch_permute(h, items) -> None:
    """Orders the union and writes every item's perm / iperm and host fields."""
    _check(lib().fp_batch_permute(h, items, len(items)), h)


def fp_batch_symbolic(h, items) -> None:
    """Every item's parent / colcount, nnzL and flops."""
    _check(lib().fp_batch_symbolic(h, items, len(items)), h)


def fp_batch_autotune(items, opts: fp_options | None = None) -> list[int]:
    opts = opts or fp_default_options()
    caps = (ctypes.c_int32 * 5)()
    _check(lib().fp_batch_autotune(items, len(items), ctypes.byref(opts), caps))
    return list(caps)


def make_batch(faces_list, n_list, caps=None, outputs=True, dof: int = 1):
    """Builds a ctypes array of fp_batch_item for CUDA face tensors, with fresh
    CUDA output tensors (kept alive on the returned object as .tensors)."""
    import torch
    items = (fp_batch_item * len(faces_list))()
    keep = []
    for i, (f, n) in enumerate(zip(faces_list, n_list)):
        it = items[i]
        it.d_faces = f.data_ptr() if f.shape[0] else None
        it.n_faces = int(f.shape[0])
        it.n_vertices = int(n)
        it.patch_cap = int(caps[i]) if caps is not None else 0
        outs = None
        if outputs:
            outs = [torch.empty(max(n * dof, 1), dtype=torch.int32, device=f.device) for _ in range(4)]
            it.d_perm, it.d_iperm, it.d_parent, it.d_colcount = [o.data_ptr() for o in outs]
        keep.append((f, outs))
    items.tensors = keep
    return items


# ---- convenience wrapper ---------------------------------------------------------

@dataclass
class Result:
    perm: object
    iperm: object
    parent: object
    colcount: object
    nnzL: int
    flops: int
    k: int
    depth: int
    gmap: object
    node_of: object
    node_begin: object
    node_size: object
    launches: int


# ---- a10 learned priorities -------------------------------------------------------

GNN_NPARAMS = 2529
GNN_FIELDS = (("w1s", (32, 6)), ("w1n", (32, 6)), ("b1", (32,)), ("w2s", (32, 32)), ("w2n", (32, 32)),
              ("b2", (32,)), ("w3", (32,)), ("c", ()))


def pack_params(d: dict, dtype=None):
    """Network parameters by name -> the flat FP_GNN_NPARAMS layout."""
    import numpy as np
    parts = [np.asarray(d[k]).reshape(-1) for k, _ in GNN_FIELDS]
    flat = np.concatenate(parts)
    assert flat.size == GNN_NPARAMS
    return flat.astype(dtype or flat.dtype)


def unpack_params(flat) -> dict:
    import numpy as np
    flat = np.asarray(flat)
    out, o = {}, 0
    for k, sh in GNN_FIELDS:
        size = int(np.prod(sh)) if sh else 1
        out[k] = flat[o:o + size].reshape(sh) if sh else flat[o]
        o += size
    return out


def fp_set_priority_net(h, codes=None):
    """codes: FP_GNN_NPARAMS int32 codes (numpy), or None to detach."""
    import numpy as np
    if codes is None:
        _check(lib().fp_set_priority_net(h, None), h)
        return
    c = np.ascontiguousarray(codes, dtype=np.int32)
    assert c.size == GNN_NPARAMS
    _check(lib().fp_set_priority_net(h, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), h)


def fp_learned_stats(h) -> tuple[int, int, int, int]:
    a, b = ctypes.c_int32(), ctypes.c_int32()
    c, d = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().fp_learned_stats(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)), h)
    return a.value, b.value, c.value, d.value


def fp_gnn_scores(h, codes, scores=None, features=None):
    import numpy as np
    c = np.ascontiguousarray(codes, dtype=np.int32)
    assert c.size == GNN_NPARAMS
    _check(lib().fp_gnn_scores(h, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _ptr(scores), _ptr(features)), h)


@dataclass
class Sample:
    """Training sample of one plain ordering (device tensors, per position)."""
    n: int
    x: object         # uint8 [n*8] feature codes
    mask: object      # uint8 [n]
    target: object    # float32 [n]
    rank: object      # int32 [n]
    lrowptr: object   # int32 [n+1]
    lcol: object      # int32 [nnz]


def fp_gnn_sample(h, n_seeds: int = 8) -> Sample:
    import torch
    n, _b, nnz = fp_get_sizes(h)
    dev = torch.device("cuda", torch.cuda.current_device())
    x = torch.zeros(max(n, 1) * 8, dtype=torch.uint8, device=dev)
    mask = torch.zeros(max(n, 1), dtype=torch.uint8, device=dev)
    target = torch.zeros(max(n, 1), dtype=torch.float32, device=dev)
    rank = torch.zeros(max(n, 1), dtype=torch.int32, device=dev)
    lrp = torch.zeros(n + 1, dtype=torch.int32, device=dev)
    lcol = torch.zeros(max(nnz, 1), dtype=torch.int32, device=dev)
    used = ctypes.c_int64()
    _check(lib().fp_gnn_sample(h, n_seeds, _ptr(x), _ptr(mask), _ptr(target), _ptr(rank), _ptr(lrp), _ptr(lcol),
                               max(nnz, 1), ctypes.byref(used)), h)
    return Sample(n, x, mask, target, rank, lrp, lcol[:used.value])


def gnn_work(n: int):
    import torch
    return torch.empty(int(lib().fp_gnn_train_work_bytes(int(n))), dtype=torch.uint8, device="cuda")


def fp_gnn_train_step(params, grad, sample: Sample, lr: float, loss, work, stream=None):
    """params/grad: float32 CUDA [FP_GNN_NPARAMS]; loss: float32 CUDA [1]."""
    _check(lib().fp_gnn_train_step(_ptr(params), _ptr(grad), _ptr(sample.x), _ptr(sample.mask),
                                   _ptr(sample.target), _ptr(sample.lrowptr), _ptr(sample.lcol), sample.n,
                                   float(lr), _ptr(loss), _ptr(work), work.numel(), _stream(stream)))


def fp_gnn_quantise(params, codes, stream=None):
    _check(lib().fp_gnn_quantise(_ptr(params), _ptr(codes), _stream(stream)))


def order_faces(faces, n_vertices: int, stream=None, symbolic: bool = True, net=None, gmap=None, k=None,
                **opt) -> Result:
    """Create + permute (+ symbolic) for a CUDA face tensor; returns every output
    as CUDA tensors (perm/iperm/parent/colcount at DOF level, the rest at
    vertex level). net: optional priority-network codes (learned leaf orders);
    gmap, k: optional supplied patches (fp_set_patches)."""
    import torch
    o = fp_default_options(**opt)
    h = fp_create_from_faces(faces, n_vertices, o, stream)
    try:
        if net is not None:
            fp_set_priority_net(h, net)
        if gmap is not None:
            fp_set_patches(h, gmap, k)
        return _run(h, n_vertices, o, stream, symbolic)
    finally:
        fp_destroy(h)


def order_csr(rowptr, col, n_rows: int, stream=None, symbolic: bool = True, gmap=None, k=None, **opt) -> Result:
    o = fp_default_options(**opt)
    h = fp_create_from_csr(rowptr, col, n_rows, o, stream)
    try:
        if gmap is not None:
            fp_set_patches(h, gmap, k)
        return _run(h, n_rows // o.dof_per_vertex, o, stream, symbolic)
    finally:
        fp_destroy(h)


def _run(h, n, o, stream, symbolic) -> Result:
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    N = n * o.dof_per_vertex
    i32 = dict(dtype=torch.int32, device=dev)
    perm = torch.empty(max(N, 1), **i32)
    iperm = torch.empty(max(N, 1), **i32)
    fp_permute(h, perm, iperm)
    parent = colcount = None
    nnz = fl = 0
    if symbolic:
        parent = torch.empty(max(N, 1), **i32)
        colcount = torch.empty(max(N, 1), **i32)
        nnz, fl = fp_symbolic(h, parent, colcount)
        parent, colcount = parent[:N], colcount[:N]
    depth = fp_get_tree(h)
    nn = (1 << (depth + 1)) - 1
    nb = torch.empty(nn, **i32)
    ns = torch.empty(nn, **i32)
    nod = torch.empty(max(n, 1), **i32)
    fp_get_tree(h, nb, ns, nod)
    gmap = torch.empty(max(n, 1), **i32)
    k = fp_get_patches(h, gmap)
    torch.cuda.current_stream().synchronize() if stream is None else torch.cuda.synchronize()
    return Result(perm[:N], iperm[:N], parent, colcount, nnz, fl, k, depth, gmap[:n], nod[:n], nb, ns,
                  fp_launch_count(h))
