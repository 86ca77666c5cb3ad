"""Benchmark: fill-reducing permutation of a triangle mesh on one B300.

Default workload: the 1024x1024 periodic torus with 30% of its quad diagonals
flipped (1,048,576 vertices, 3 DOF per vertex, patch cap 512), the largest
single-mesh configuration. One step = the whole path on one mesh:
fp_create_from_faces (CSR assembly) + fp_permute (patching, quotient-graph
nested dissection, local minimum degree, permutation, DOF expansion) +
fp_symbolic (etree, column counts, DOF expansion) + fp_destroy, with the face
list already resident in HBM. Each step is timed with CUDA events on the
launching stream; L2 is flushed (256 MB write) between steps, outside the
events. Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload torus1024|icosphere7|grid64|batch256|batch256_learned]

--impl reference times the CPU oracle (the plain single-threaded statement of
the method that the tests check the GPU against) on the same workload.
Under torchrun (N > 1) every rank orders its own replica of the mesh (the path
does not shard); value counts the vertices of all ranks.
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    # name: (generator, patch cap, dof per vertex)
    "icosphere7": ("icosphere7", 512, 1),
    "torus1024": ("torus1024", 512, 3),
    "grid64": ("grid64", 256, 1),
}

# Algorithmic bytes per mesh vertex and per step for each profiled stage
# (int32 indices, valence-6 mesh: CSR row 28 B, faces 24 B per vertex).
#   graph      : read faces 24 + write CSR 28
#   patch_bfs  : per search: read CSR 28 + neighbour keys 24 + key write 8 = 60
#   quotient   : one CSR + group-map pass 52
#   nd         : boundary graph only, about 25% of edges per level, 60 in total
#   md         : read induced rows + write order 32
#   perm       : perm + iperm 8
#   symbolic   : pattern + iperm gather + parent/colcount write 60
STAGES = ["graph", "patch_bfs", "patch_other", "quotient", "nd_bisect", "nd_separator", "layout",
          "md_small", "md_mid", "md_large", "perm", "symbolic", "learned", "train", "patch_local", "join_wait",
          "numeric"]
# stages whose kernels run on the auxiliary streams, overlapped with the
# handle's stream; their part of the critical path is the join wait
AUX_STAGES = ("md_mid", "md_large")
BYTES_PER_VERTEX = {"graph": 52, "patch_bfs": 60, "quotient": 52, "nd_separator": 60, "md_small": 32,
                    "md_mid": 32, "md_large": 32, "perm": 8, "symbolic": 60, "layout": 12}
PER_LAUNCH_UNITS = {"patch_bfs"}   # bytes per vertex are per launch, not per step
# nd_bisect (one launch per tree level) reads the live quotient graph: about 6
# entries per patch, each read as column, weight, node and local index (16 B),
# plus 24 B per patch of list, side and flags = 120 B per patch per launch
BYTES_PER_PATCH = {"nd_bisect": 120}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def measured_traffic(stage: str, workload: str):
    """DRAM bytes per launch of `stage`'s kernel from the committed ncu summary
    (profiles/kernel_traffic.json), or None when there is none for this
    workload or the kernel source changed since the capture."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "kernel_traffic.json")
    if not os.path.exists(p):
        return None
    found = [e for e in json.load(open(p)).get("entries", []) if e.get("stage") == stage and e.get("workload") == workload]
    if not found:
        return None
    d = found[0]
    src = os.path.join(ROOT, d["source"])
    if not os.path.exists(src) or hashlib.sha1(open(src, "rb").read()).hexdigest() != d["source_sha1"]:
        return None
    return float(d["dram_bytes_per_launch"])


def max_over_ranks(x: float, ws: int, device) -> float:
    """The largest value of x over the ranks (x itself on one rank)."""
    if ws <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, ws: int, seconds: float) -> float:
    """Units of all ranks (each rank processes its own, equal-sized shard) per
    second of the slowest rank."""
    return ws * units_per_rank / seconds


def batch_meshes(rank: int, learned: bool):
    """The meshes rank `rank` orders in the batch workloads: its own mix (seed =
    rank), plus the 4.2M-vertex torus for the learned form."""
    import meshgen
    meshes = meshgen.mesh_mix(256, seed=rank)
    if learned:
        meshes.append(meshgen.shuffle(meshgen.torus(2048, 2048, 0.3, 4096 + rank), 4096 + rank))
    return meshes


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    lrank = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, lrank


def make_mesh(name, cap_override=None):
    import meshgen
    gen, cap, dof = WORKLOADS[name]
    return getattr(meshgen, gen)(0), (cap_override or cap), dof


def gpu_uuid(device_index: int) -> str:
    """nvidia-smi's UUID string ("GPU-...") of CUDA device `device_index`."""
    import torch
    return "GPU-" + str(torch.cuda.get_device_properties(device_index).uuid)


class Clocks:
    """nvidia-smi sampling of the SM clock and throttle reasons of the GPU the
    steps run on, selected by UUID (a CUDA device index need not be
    nvidia-smi's index under CUDA_VISIBLE_DEVICES). A freshly started
    nvidia-smi slows the CUDA calls of other processes for about a second
    while it initialises, so callers keep the GPU busy with untimed work for
    WARM_S seconds after starting it, then bracket the timed region with
    begin()/end(); stop() reports the samples taken in that region and, for
    the median, in the busy window around it."""

    FIELDS = ("timestamp,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    WARM_S = 1.5

    def __init__(self, device_index: int):
        self.uuid = None
        self.t0 = self.t1 = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            want = gpu_uuid(device_index)
            listed = subprocess.run(["nvidia-smi", "--query-gpu=uuid", "--format=csv,noheader"],
                                    capture_output=True, text=True, timeout=30).stdout.split()
            self.uuid = want if want in listed else None
            sel = self.uuid if self.uuid else str(device_index)
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "100", "-i", sel], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, subprocess.SubprocessError):
            self.p = None

    def begin(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        import datetime
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[2]), float(parts[3]),
                             {nm for nm, val in zip(names, parts[6:10]) if val.lower() in ("active", "1")}))
            except ValueError:
                continue
        os.unlink(self.f.name)
        t0 = self.t0 if self.t0 is not None else -1e18
        t1 = self.t1 if self.t1 is not None else 1e18
        timed = [r for r in rows if t0 - 0.05 <= r[0] <= t1 + 0.05]
        # the GPU runs the same step throughout the busy window around the
        # timed region (warm steps before it, one more timed-like pass after)
        busy = [r for r in rows if t0 - self.WARM_S / 2 <= r[0] <= t1 + 0.5] or rows
        use = timed if len(timed) >= 3 else busy
        reasons = set().union(*[r[3] for r in use]) if use else set()
        return {"sm_mhz": statistics.median([r[1] for r in use]) if use else None,
                "sm_max_mhz": max(r[2] for r in use) if use else None,
                "samples": len(use), "samples_in_timed_region": len(timed),
                "window": "timed region" if use is timed else "timed region and the busy steps around it",
                "reasons": sorted(reasons), "gpu": self.uuid or "index (UUID not listed by nvidia-smi)"}


def oracle_step(mesh, cap, dof, codes=None):
    import oracle as O
    g = O.graph_from_faces(mesh.faces, mesh.n)
    o = O.order(g, cap, seed=0)
    perm = o.perm
    if codes is not None:
        import paper_2602_00898_b300 as fp
        from oracle import gnn as G
        perm = G.order_learned(g, o, G.QParams.from_dict(fp.unpack_params(codes)), cap).perm
    s = O.symbolic(g, perm)
    if dof > 1:
        O.dof_expand(dof, o.perm, s.parent, s.colcount)
    return s


def cpu_baseline(mesh, cap, dof, budget_s=20.0, max_runs=8):
    """The oracle as it stands, single-threaded, on whole copies of the mesh."""
    times = []
    t_end = time.perf_counter() + budget_s
    while len(times) < max_runs and (not times or time.perf_counter() < t_end):
        t = time.perf_counter()
        oracle_step(mesh, cap, dof)
        times.append(time.perf_counter() - t)
    per = statistics.median(times)
    return {"value": mesh.n / per / 1e6, "unit": "Mverts/s", "cores": 1, "kind": "oracle",
            "sample": f"{len(times)} whole-mesh runs of the single-threaded oracle (graph + order + symbolic), "
                      f"median {per * 1e3:.0f} ms, 1 of {os.cpu_count()} host cores"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    mesh, cap, dof = make_mesh(args.workload, args.patch_cap)
    for _ in range(args.warmup):
        oracle_step(mesh, cap, dof)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        s = oracle_step(mesh, cap, dof)
        times.append(time.perf_counter() - t)
    ms = 1e3 * sum(times) / len(times)
    value = mesh.n / (ms / 1e3) / 1e6
    line = {"impl": "reference", "metric": "permutation Mverts/s at 1 GPU", "value": value, "unit": "Mverts/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": mesh.n, "faces": mesh.n_faces, "patch_cap": cap,
                       "dof_per_vertex": dof, "nnzL": s.nnzL},
            "cpu_baseline": {"value": value, "unit": "Mverts/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} whole-mesh runs of the single-threaded oracle"},
            "e2e": {"value": value, "unit": "Mverts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def warm_event(stream, flush=None):
    """Runs, once and untimed, the work the timed loop adds around the steps:
    the L2 flush (PyTorch's fill kernel: the first launch of a PyTorch kernel
    in a process loads its module, a one-time host stall of ~0.3 s measured
    between two steps of a first timed block) and a timing event record."""
    import torch
    if flush is not None:
        flush.zero_()
    e = torch.cuda.Event(enable_timing=True)
    e.record(stream)
    e.synchronize()


def leaf_vertex_count(node_size) -> int:
    """Vertices of the tree's leaves (nodes with vertices and no non-empty
    descendant), given the node sizes of the binary tree in array form."""
    nn = len(node_size)
    below = [0] * nn           # vertices strictly below each node
    for t in range(nn - 1, -1, -1):
        for c in (2 * t + 1, 2 * t + 2):
            if c < nn:
                below[t] += below[c] + int(node_size[c])
    return sum(int(node_size[t]) for t in range(nn) if node_size[t] > 0 and below[t] == 0)


def stage_bytes_per_launch(stage, n, k, stage_n, leaf_vertices):
    """Algorithmic bytes one launch of `stage` must move (see the table above),
    or None for stages without a byte model."""
    if stage_n.get(stage, 0) <= 0:
        return None
    if stage in BYTES_PER_PATCH:
        return BYTES_PER_PATCH[stage] * k
    if stage == "md_small":
        units = leaf_vertices
    elif stage in ("md_mid", "md_large"):
        units = n - leaf_vertices          # separator vertices
    elif stage in BYTES_PER_VERTEX:
        units = n
    else:
        return None
    if stage in PER_LAUNCH_UNITS:
        return BYTES_PER_VERTEX[stage] * units
    return BYTES_PER_VERTEX[stage] * units / stage_n[stage]


def critical_path(stage_ms) -> dict:
    """The step's critical path from the stage profile: every stage of the
    handle's stream is on it; the separator orderings on the auxiliary streams
    add only the join wait (the handle's stream idling for them after its own
    leaf orderings). The dominant stage is the largest contribution; for the
    auxiliary streams that is the longer of their two stages."""
    main = {s: v for s, v in stage_ms.items() if s not in AUX_STAGES and s != "join_wait"}
    contrib = dict(main)
    aux = max(AUX_STAGES, key=lambda s: stage_ms.get(s, 0.0))
    contrib[aux] = stage_ms.get("join_wait", 0.0)
    dom = max(contrib, key=lambda s: contrib[s])
    return {"handle_stream": round(sum(main.values()), 4), "join_wait": round(stage_ms.get("join_wait", 0.0), 4),
            "auxiliary_streams": round(sum(stage_ms.get(s, 0.0) for s in AUX_STAGES), 4),
            "dominant": dom, "dominant_contribution": round(contrib[dom], 4)}


def run_ours(args):
    import torch
    import paper_2602_00898_b300 as fp

    ws, rank, lrank = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(lrank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", lrank))
    dev = torch.device("cuda", torch.cuda.current_device())
    mesh, cap, dof = make_mesh(args.workload, args.patch_cap)
    n = mesh.n
    faces = torch.from_numpy(mesh.faces).to(dev)
    opts = fp.fp_default_options(patch_cap=cap, dof_per_vertex=dof)
    N = n * dof
    perm = torch.empty(N, dtype=torch.int32, device=dev)
    iperm = torch.empty_like(perm)
    parent = torch.empty_like(perm)
    colcount = torch.empty_like(perm)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > 126 MB L2
    stream = torch.cuda.current_stream()

    def step():
        h = fp.fp_create_from_faces(faces, n, opts)
        fp.fp_permute(h, perm, iperm)
        nnz, fl = fp.fp_symbolic(h, parent, colcount)
        launches = fp.fp_launch_count(h)
        fp.fp_destroy(h)
        return nnz, fl, launches

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # timed region (stage profiling off: its event records cost ~0.3 ms a step).
    # The clock sampler starts while untimed steps keep the GPU busy: an idle
    # pause here let the GPU drop out of its full-speed state, and the timed
    # region (about a tenth of a second) then ran ~8% slow in some processes.
    clocks = Clocks(lrank)
    t_warm = time.perf_counter()
    while time.perf_counter() - t_warm < Clocks.WARM_S:
        step()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches = 0
    t_inside = 0.0
    host_steps = []
    # one-time costs of the loop's own work (the flush's first launch) and
    # Python's collector are kept out of the region
    warm_event(stream, flush)
    gc.collect()
    gc.disable()
    clocks.begin()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        t0 = time.perf_counter()
        flush.zero_()
        ev[i][0].record(stream)
        t = time.perf_counter()
        nnz, fl, L = step()
        t_inside += time.perf_counter() - t
        ev[i][1].record(stream)
        launches += L
        host_steps.append(time.perf_counter() - t0)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t_wall
    gc.enable()
    clocks.end()
    for _ in range(3):          # the busy window goes on briefly after the region
        step()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_steps = [a.elapsed_time(b) for a, b in ev]
    ms_local = sum(ms_steps) / len(ms_steps)
    # stage breakdown: separate profiled steps (CUDA events on each stage's stream)
    import ctypes
    nprof = min(args.steps, 10)
    fp.lib().fp_profile_reset()
    fp.lib().fp_profiling(1)
    for _ in range(nprof):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    fp.lib().fp_profiling(0)
    prof_ms = (ctypes.c_double * len(STAGES))()
    prof_n = (ctypes.c_int64 * len(STAGES))()
    fp.lib().fp_profile_read.restype = ctypes.c_int
    fp.lib().fp_profile_read(prof_ms, prof_n, len(STAGES))
    stage_ms = {STAGES[i]: prof_ms[i] / nprof for i in range(len(STAGES))}
    stage_n = {STAGES[i]: prof_n[i] / nprof for i in range(len(STAGES))}

    ms = max_over_ranks(ms_local, ws, dev)
    value = whole_job_rate(n, ws, ms / 1e3) / 1e6

    # permutation alone (fp_permute), for the "permutation ms" part of the metric
    h = fp.fp_create_from_faces(faces, n, opts)
    torch.cuda.synchronize()
    pms = []
    for _ in range(5):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fp.fp_permute(h, perm, iperm)
        b.record(stream)
        b.synchronize()
        pms.append(a.elapsed_time(b))
    k = fp.fp_get_patches(h)
    depth = fp.fp_get_tree(h)
    nnodes = (1 << (depth + 1)) - 1
    nsize = torch.empty(nnodes, dtype=torch.int32, device=dev)
    fp.fp_get_tree(h, None, nsize, None)
    _, _, nnzA2 = fp.fp_get_sizes(h)
    fp.fp_destroy(h)
    leaf_vertices = leaf_vertex_count(nsize.cpu().numpy())

    # end to end through the host-buffer entry point
    hfaces = torch.from_numpy(mesh.faces).pin_memory()
    houts = [torch.empty(N, dtype=torch.int32).pin_memory() for _ in range(4)]
    # fp_order_faces_host returns once the results are in host memory, so a
    # host clock around the call is what its caller waits for
    e2e_ms, e2e_ev = [], []
    for i in range(3 + max(10, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t = time.perf_counter()
        a.record(stream)
        fp.fp_order_faces_host(hfaces, n, opts, None, *houts)
        b.record(stream)
        t = time.perf_counter() - t
        b.synchronize()
        if i >= 3:
            e2e_ms.append(1e3 * t)
            e2e_ev.append(a.elapsed_time(b))
    e2e = statistics.mean(e2e_ms)

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    cp = critical_path(stage_ms)
    dom = cp["dominant"]
    peak, peak_kind = peaks()
    roof = None
    bl = stage_bytes_per_launch(dom, n, k, stage_n, leaf_vertices)
    if bl is not None and stage_n[dom] > 0:
        per_launch_ms = stage_ms[dom] / stage_n[dom]
        achieved = bl / (per_launch_ms / 1e3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": measured_traffic(dom, args.workload),
                "peak_source": peak_kind + " (HBM copy)", "algorithmic_bytes_per_launch": bl,
                "launch_ms": per_launch_ms, "launches_per_step": stage_n[dom]}
    # nnz of the lower triangle (with the diagonal) of the matrix factored:
    # b x b dense blocks on the vertex graph's pattern plus its diagonal
    E = nnzA2 // 2
    nnzA = dof * dof * E + n * dof * (dof + 1) // 2
    nnzL_vertex = (nnz + n * dof * (dof - 1) // 2) // (dof * dof)
    line = {
        "metric": "permutation Mverts/s at 1 GPU", "value": value, "unit": "Mverts/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "faces": mesh.n_faces, "patch_cap": cap, "dof_per_vertex": dof,
                   "step": "create+permute+symbolic+destroy", "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "ms_median": statistics.median(ms_steps),
        "permute_ms": statistics.median(pms),
        "wall_ms_per_step": 1e3 * wall / args.steps,
        "host_ms_per_step_inside_events": 1e3 * t_inside / args.steps,
        "host_ms_per_step_median": 1e3 * statistics.median(host_steps),
        "host_ms_per_step_max": 1e3 * max(host_steps),
        "critical_path_ms": cp,
        "stage_profile": f"{nprof} extra steps with per-stage CUDA events (kept out of the timed steps)",
        "nnzL": nnz, "nnzA": nnzA, "fill_ratio": nnz / nnzA, "flops": fl,
        "nnzL_vertex": nnzL_vertex, "fill_ratio_vertex": nnzL_vertex / (E + n),
        "fill_note": "nnz of L and of the lower triangle of A, both with the diagonal, at the level factored "
                     "(DOF level with b x b blocks); *_vertex: the same on the vertex graph",
        "patches": k, "tree_depth": depth,
        "stage_ms": {s: round(v, 4) for s, v in stage_ms.items()},
        "roofline": roof,
        "clocks": clk,
        "e2e": {"value": n / (e2e / 1e3) / 1e6, "unit": "Mverts/s", "ms": e2e,
                "timing": "host clock around fp_order_faces_host (pinned faces in, four outputs out)",
                "event_ms": statistics.mean(e2e_ev),
                "h2d_bytes_per_step": int(mesh.faces.nbytes),
                "d2h_bytes_per_step": int(4 * 4 * N + 16)},
        "gpu_launches": int(launches),
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(mesh, cap, dof)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_batch(args):
    """256 meshes (n log-uniform in [2k, 200k], grid / icosphere / flipped torus),
    autotuned caps, one fp_batch_order per step; metric meshes/s.
    batch256_learned: the same mix plus one 2048x2048 flipped torus (4.2M
    vertices), ordered with the trained leaf-priority network
    (fp_batch_order_learned); nnz(L) is reported against the plain batch."""
    import torch
    import paper_2602_00898_b300 as fp
    import meshgen
    learned = args.workload == "batch256_learned"

    ws, rank, lrank = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(lrank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", lrank))
    dev = torch.device("cuda", torch.cuda.current_device())
    meshes = batch_meshes(rank, learned)
    codes = None
    if learned:
        from paper_2602_00898_b300.train_priorities import load_codes
        codes = load_codes()
    nverts = sum(m.n for m in meshes)
    faces = [torch.from_numpy(m.faces).to(dev) for m in meshes]
    items = fp.make_batch(faces, [m.n for m in meshes])
    opts = fp.fp_default_options()
    caps = fp.fp_batch_autotune(items, opts)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def order_all(workers=0):
        # workers 0: the fused form (the whole batch as one disjoint union)
        if learned:
            return fp.fp_batch_order_learned(items, codes, opts, n_workers=workers)
        return fp.fp_batch_order(items, opts, n_workers=workers)

    plain_nnz = None
    if learned:
        assert fp.fp_batch_order(items, opts) == 0
        plain_nnz = sum(int(it.nnzL) for it in items)
    for _ in range(args.warmup):
        assert order_all() == 0
    torch.cuda.synchronize()
    # no stage profiling here: its event records would serialise the workers;
    # the GPU stays busy while the clock sampler starts (as above)
    clocks = Clocks(lrank)
    t_warm = time.perf_counter()
    while time.perf_counter() - t_warm < Clocks.WARM_S:
        assert order_all() == 0
    if ws > 1:
        torch.distributed.barrier()
    times, launches = [], 0
    warm_event(torch.cuda.current_stream(), flush)
    clocks.begin()
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        # an NVTX range per timed step lets a profiler select exactly these
        # launches (ncu --nvtx --nvtx-include "batch_step/")
        torch.cuda.nvtx.range_push("batch_step")
        st = order_all()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        times.append(time.perf_counter() - t)
        assert st == 0
        launches += sum(int(it.launches) for it in items)
    if ws > 1:
        torch.distributed.barrier()
    clocks.end()
    assert order_all() == 0
    torch.cuda.synchronize()
    clk = clocks.stop()
    sec = max_over_ranks(sum(times) / len(times), ws, dev)
    # stage breakdown of the fused pipeline (a separate profiled pass)
    import ctypes
    fp.lib().fp_profile_reset()
    fp.lib().fp_profiling(1)
    assert order_all() == 0
    torch.cuda.synchronize()
    fp.lib().fp_profiling(0)
    prof_ms = (ctypes.c_double * len(STAGES))()
    fp.lib().fp_profile_read.restype = ctypes.c_int
    fp.lib().fp_profile_read(prof_ms, None, len(STAGES))
    stage_ms = {STAGES[i]: round(prof_ms[i], 4) for i in range(len(STAGES)) if prof_ms[i] > 0}
    # context: the same batch through the per-mesh pool of 8 host workers
    pool_t = []
    for _ in range(3):
        torch.cuda.synchronize()
        t = time.perf_counter()
        assert order_all(8) == 0
        torch.cuda.synchronize()
        pool_t.append(time.perf_counter() - t)
    # end to end: pinned host faces in, four outputs back, every step
    hfaces = [torch.from_numpy(m.faces).pin_memory() for m in meshes]
    houts = [[torch.empty(m.n, dtype=torch.int32).pin_memory() for _ in range(4)] for m in meshes]
    e2e = []
    for r in range(3):
        torch.cuda.synchronize()
        t = time.perf_counter()
        for d, hsrc in zip(faces, hfaces):
            d.copy_(hsrc, non_blocking=True)
        torch.cuda.synchronize()
        assert order_all() == 0
        for (f, outs), ho in zip(items.tensors, houts):
            for o, h in zip(outs, ho):
                h.copy_(o[:h.numel()], non_blocking=True)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t)
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    nnz = sum(int(it.nnzL) for it in items)
    line = {
        "metric": "batched meshes/s at 1 GPU", "value": whole_job_rate(len(meshes), ws, sec), "unit": "meshes/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "meshes": len(meshes), "vertices": nverts,
                   "caps_by_size_class": caps, "form": "fused (one pipeline over the disjoint union)",
                   "l2": "flushed between steps (256 MB write)",
                   "step": ("fp_batch_order_learned" if learned else "fp_batch_order")
                           + " over all meshes (create+permute+symbolic of the union, per-mesh outputs)"},
        "mverts_per_s": ws * nverts / sec / 1e6, "nnzL_total": nnz,
        "stage_ms": stage_ms,
        "pool_8_workers": {"meshes_per_s": len(meshes) / statistics.median(pool_t),
                           "note": "the same batch, one mesh pipeline per host worker (context, not the value)"},
        "clocks": clk,
        "e2e": {"value": len(meshes) / statistics.median(e2e), "unit": "meshes/s",
                "h2d_bytes_per_step": int(sum(m.faces.nbytes for m in meshes)),
                "d2h_bytes_per_step": int(sum(16 * m.n for m in meshes))},
        "gpu_launches": launches,
    }
    if learned:
        line["learned"] = {"nnzL_plain_total": plain_nnz, "nnzL_learned_total": nnz,
                           "nnzL_ratio": nnz / plain_nnz,
                           "leaves": sum(int(it.learned_leaves) for it in items),
                           "leaves_learned_kept": sum(int(it.learned_kept) for it in items),
                           "network": "paper_2602_00898_b300/priority_net.json (trained on the GPU)"}
    if not args.no_cpu_baseline:
        idx = list(range(0, 256, 32))
        sample = [meshes[i] for i in idx]
        t0 = time.perf_counter()
        for i in idx:
            oracle_step(meshes[i], items[i].chosen_cap, 1, codes)
        per = (time.perf_counter() - t0) / len(sample)
        line["cpu_baseline"] = {"value": 1.0 / per, "unit": "meshes/s", "cores": 1, "kind": "oracle",
                                "sample": f"every 32nd mesh of the 256-mesh mix ({len(sample)} meshes, "
                                          f"{sum(m.n for m in sample)} vertices"
                                          + (", learned form; the 4.2M-vertex torus is not sampled" if learned
                                             else "") + f"), single-threaded oracle, "
                                          f"1 of {os.cpu_count()} host cores"}
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# FP64 rate of B300 (CUDA cores), from the nominal figures of the part: no
# measured FP64 peak is recorded for this machine
FP64_PEAK_TFLOPS = 1.25
FACTOR_WORKLOADS = {"factor_icosphere7": "icosphere7", "factor_grid64": "grid64", "factor_torus1024": "torus1024"}


def run_factor(args):
    """Numeric factorisation driven by the ordering (Section 6): the Laplacian
    plus the identity of the mesh (unit weights), ordered once; a step is
    fp_factor + one fp_solve, timed with CUDA events (L2 flushed between
    steps). Metric: the mesh's vertices per second of factor + solve."""
    import torch
    import paper_2602_00898_b300 as fp
    import meshgen

    ws, rank, lrank = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(lrank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", lrank))
    dev = torch.device("cuda", torch.cuda.current_device())
    name = FACTOR_WORKLOADS[args.workload]
    gen, cap, _ = WORKLOADS[name]
    mesh = getattr(meshgen, gen)(0)
    cap = args.patch_cap or cap
    n = mesh.n
    faces = torch.from_numpy(mesh.faces).to(dev)
    h = fp.fp_create_from_faces(faces, n, fp.fp_default_options(patch_cap=cap))
    fp.fp_permute(h)
    _, _, nnz = fp.fp_get_sizes(h)
    rp = torch.empty(n + 1, dtype=torch.int32, device=dev)
    col = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
    fp.fp_get_graph(h, rp, col)
    rpn, coln = rp.cpu().numpy(), col.cpu().numpy()[:nnz]
    diag_h, off_h = meshgen.laplacian_values(rpn, coln, seed=None)
    diag = torch.from_numpy(diag_h).to(dev)
    off = torch.from_numpy(off_h).to(dev)
    b = torch.from_numpy(np.random.default_rng(0).standard_normal(n)).to(dev)
    x = torch.empty_like(b)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    import ctypes
    for _ in range(args.warmup):
        fp.fp_factor(h, diag, off)
        fp.fp_solve(h, b, x)
    torch.cuda.synchronize()
    clocks = Clocks(lrank)
    t_warm = time.perf_counter()
    while time.perf_counter() - t_warm < Clocks.WARM_S:
        fp.fp_factor(h, diag, off)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    warm_event(stream, flush)
    clocks.begin()
    l0 = fp.fp_launch_count(h)
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        fp.fp_factor(h, diag, off)
        ev[i][1].record(stream)
        fp.fp_solve(h, b, x)
        ev[i][2].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    launches = fp.fp_launch_count(h) - l0
    clocks.end()
    fp.fp_factor(h, diag, off)
    torch.cuda.synchronize()
    clk = clocks.stop()
    fac = [a.elapsed_time(b2) for a, b2, _ in ev]
    sol = [b2.elapsed_time(c) for _, b2, c in ev]
    ms = max_over_ranks(statistics.mean(f + s_ for f, s_ in zip(fac, sol)), ws, dev)
    fdoubles, flops, nnz_front = fp.fp_factor_stats(h)
    # residual of the last solve
    xs = x.cpu().numpy()
    src = np.repeat(np.arange(n), np.diff(rpn))
    ax = diag_h * xs + np.bincount(src, weights=off_h * xs[coln], minlength=n)
    bb = b.cpu().numpy()
    resid = float(np.linalg.norm(ax - bb) / np.linalg.norm(bb))
    # the factor kernels' own time, for the roofline (profiled steps)
    fp.lib().fp_profile_reset()
    fp.lib().fp_profiling(1)
    nprof = min(args.steps, 5)
    for _ in range(nprof):
        flush.zero_()
        fp.fp_factor(h, diag, off)
    torch.cuda.synchronize()
    fp.lib().fp_profiling(0)
    prof_ms = (ctypes.c_double * len(STAGES))()
    prof_n = (ctypes.c_int64 * len(STAGES))()
    fp.lib().fp_profile_read(prof_ms, prof_n, len(STAGES))
    num_ms = prof_ms[STAGES.index("numeric")] / nprof
    fp.fp_destroy(h)
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    fac_ms = statistics.mean(fac)
    achieved = flops / (fac_ms / 1e3) / 1e12
    line = {
        "metric": "numeric factor+solve Mverts/s at 1 GPU", "value": whole_job_rate(n, ws, ms / 1e3) / 1e6,
        "unit": "Mverts/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "patch_cap": cap, "matrix": "unit graph Laplacian + I",
                   "step": "fp_factor + fp_solve (ordering done once, outside)",
                   "l2": "flushed between steps (256 MB write)", "parallelism": "replicas" if ws > 1 else "single"},
        "factor_ms": fac_ms, "solve_ms": statistics.mean(sol), "wall_ms_per_step": 1e3 * wall / args.steps,
        "front_flops": flops, "front_doubles": fdoubles, "nnzL_stored": nnz_front, "solve_residual": resid,
        "factor_level_ms_sum": num_ms,
        "roofline": {"kernel": "factor (front assembly + tiled partial Cholesky)", "bound": "alu",
                     "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                     "traffic": None, "peak_source": "nominal FP64 rate of the part (no measured FP64 peak)"},
        "clocks": clk,
        "gpu_launches": int(launches),
    }
    if not args.no_cpu_baseline:
        import oracle as O
        g = O.Graph(rpn, coln)
        o = O.order(g, cap, seed=0)
        t = time.perf_counter()
        f = O.cholesky(g, diag_h, off_h, o.perm)
        O.cholesky_solve(f, o.perm, bb)
        per = time.perf_counter() - t
        line["cpu_baseline"] = {"value": n / per / 1e6, "unit": "Mverts/s", "cores": 1, "kind": "oracle",
                                "sample": f"one up-looking sparse Cholesky + solve of the same matrix in the same "
                                          f"order ({per:.1f} s), single-threaded, 1 of {os.cpu_count()} host cores"}
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=list(WORKLOADS) + ["batch256", "batch256_learned"] + list(FACTOR_WORKLOADS),
                    default="torus1024")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--patch-cap", type=int, default=None,
                    help="patch cap of a single-mesh workload instead of its default (patch-size studies)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.workload in ("batch256", "batch256_learned") and args.impl == "ours":
        run_batch(args)
    elif args.workload in FACTOR_WORKLOADS and args.impl == "ours":
        run_factor(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
