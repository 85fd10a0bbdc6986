"""The multi-rank (N > 1) host logic of the benchmark on CPU with the gloo
backend and two ranks: walkers are sharded (each rank evaluates its own,
distinct batch; no collective on the data path), the step time is the max over
ranks, and the reported value counts the walkers of every rank."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1510_00730_gb300 import synth
    wl = synth.oxygen_like_1k()
    batches = bench.rank_batches(wl, rank)
    sums = torch.tensor([float(np.sum(b)) for b in batches], dtype=torch.float64)
    gathered = [torch.empty_like(sums) for _ in range(world)]
    dist.all_gather(gathered, sums)
    local_ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
    ms = bench._max_over_ranks(local_ms, dist, torch.device("cpu"))
    out.put((rank, ms, bench.whole_job_value(wl.n_walk, world, ms), [g.tolist() for g in gathered],
             [b.shape for b in batches]))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, v0, g0, sh0), (r1, ms1, v1, g1, sh1) = res
    assert ms0 == ms1 == 15.0                 # max over ranks
    assert v0 == v1 == pytest.approx(2 * 64 / 0.015)   # both ranks' walkers over the slower rank's time
    assert g0 == g1                           # both ranks saw the same gathered checksums
    assert not set(g0[0]) & set(g0[1])        # the ranks' walker batches are distinct
    assert sh0 == sh1 == [(64, 8, 3)] * 4
