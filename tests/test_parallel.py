"""Multi-rank sharding on CPU ranks (torch.distributed, gloo, world size 2)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2312_13513_gb300.parallel import partition_by_weight, shard  # noqa: E402


def test_partition_tiles_and_balances():
    rng = np.random.default_rng(0)
    w = rng.integers(1, 50, 10007).astype(float)
    for world in (1, 2, 3, 8):
        parts = partition_by_weight(w, world)
        assert parts[0][0] == 0 and parts[-1][1] == w.size
        for a, b in zip(parts, parts[1:]):
            assert a[1] == b[0]
        sums = [w[s:e].sum() for s, e in parts]
        assert max(sums) - min(sums) <= 2 * w.max() + 1e-9
    assert partition_by_weight([], 2) == [(0, 0), (0, 0)]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(42)            # every rank sees the same previous-step counts
    weights = rng.integers(1, 30, n).astype(float)
    s, e = shard(n, rank, world, weights)
    # each rank reports its range and its work; no data-path collective is needed, this one only
    # checks the partition
    mine = torch.tensor([s, e, weights[s:e].sum()], dtype=torch.float64)
    gathered = [torch.zeros(3, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, mine)
    if rank == 0:
        out.put([g.tolist() for g in gathered])
    dist.destroy_process_group()


def test_two_gloo_ranks_cover_every_cell_once():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    n = 5003
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (s0, e0, w0), (s1, e1, w1) = res
    assert s0 == 0 and e0 == s1 and e1 == n
    assert abs(w0 - w1) <= 2 * 29
