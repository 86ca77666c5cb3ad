"""The N > 1 host path of bench.py on CPU: two gloo ranks check the
max-over-ranks timing, the whole-job rate and that the ranks' batch shards
are different meshes (no data-path collective exists to test)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        local = 1.0 + 0.5 * rank
        m = bench.max_over_ranks(local, ws, "cpu")
        first = bench.batch_meshes(rank, False)[0]
        sig = torch.tensor([float(first.n), float(first.faces[:64].sum())], dtype=torch.float64)
        sigs = [torch.zeros(2, dtype=torch.float64) for _ in range(ws)]
        dist.all_gather(sigs, sig)
        out[rank] = (m, bench.whole_job_rate(256, ws, m), [tuple(x.tolist()) for x in sigs])
    finally:
        dist.destroy_process_group()


def test_two_rank_host_path():
    ws = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(ws, port, out), nprocs=ws, join=True, start_method="spawn")
    for r in range(ws):
        m, rate, sigs = out[r]
        assert m == 1.5                      # the slowest rank's time
        assert rate == pytest.approx(2 * 256 / 1.5)
        assert sigs[0] != sigs[1]            # different shards
    assert out[0][2] == out[1][2]


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.25, 1, "cpu") == 3.25
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0
