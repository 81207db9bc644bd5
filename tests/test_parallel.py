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


def test_flat_gradient_layout_round_trip_and_batch_shares():
    from paper_2312_13513_gb300.parallel import batch_share, flatten_grads, unflatten_grads
    rng = np.random.default_rng(1)
    shapes = [(7, 3), (5, 7), (2, 5)]
    dW = [rng.standard_normal(s) for s in shapes]
    db = [rng.standard_normal(s[0]) for s in shapes]
    flat = flatten_grads(dW, db)
    assert flat.size == sum(r * c + r for r, c in shapes)
    # layer by layer: dW row-major, then db
    assert np.array_equal(flat[:21], dW[0].reshape(-1)) and np.array_equal(flat[21:28], db[0])
    gW, gb = unflatten_grads(flat, shapes)
    assert all(np.array_equal(a, b) for a, b in zip(gW, dW)) and all(np.array_equal(a, b) for a, b in zip(gb, db))
    with pytest.raises(ValueError):
        unflatten_grads(flat[:-1], shapes)
    idx = np.arange(12)
    assert np.array_equal(np.concatenate([batch_share(idx, r, 3) for r in range(3)]), idx)
    with pytest.raises(ValueError):
        batch_share(idx, 0, 5)


def _dp_worker(rank, world, port, out):
    """One data-parallel training step of a small GELU network with the oracle's FP64 backward on
    this rank's share of the global batch, the package's gradient all-reduce, then Adam."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import mlp as omlp
    from paper_2312_13513_gb300.parallel import allreduce_sum_, batch_share, flatten_grads, unflatten_grads
    rng = np.random.default_rng(3)                # the same network and batch on every rank
    dims = [11, 48, 48, 9]
    W = [rng.standard_normal((dims[i + 1], dims[i])) / np.sqrt(dims[i]) for i in range(3)]
    b = [0.1 * rng.standard_normal(dims[i + 1]) for i in range(3)]
    X = rng.standard_normal((64, 11))
    T = rng.standard_normal((64, 9))
    share = batch_share(np.arange(64), rank, world)
    o, cache = omlp.forward(W, b, X[share], emulate_bf16=False)
    dW, db = omlp.backward(W, b, cache, o, T[share])
    flat = torch.tensor(flatten_grads(dW, db))
    n = allreduce_sum_(flat)
    flat /= n
    gW, gb = unflatten_grads(flat.numpy(), [(dims[i + 1], dims[i]) for i in range(3)])
    # the single-rank gradient of the whole global batch
    o1, c1 = omlp.forward(W, b, X, emulate_bf16=False)
    rW, rb = omlp.backward(W, b, c1, o1, T)
    gerr = max(np.max(np.abs(a - r)) / np.max(np.abs(r)) for a, r in zip(gW + gb, rW + rb))
    params = [w.copy() for w in W] + [x.copy() for x in b]
    zeros = [np.zeros_like(x) for x in params]
    p_dp, _, _ = omlp.adam_step([x.copy() for x in params], gW + gb, [z.copy() for z in zeros],
                                [z.copy() for z in zeros], 1, lr=1e-3)
    p_1, _, _ = omlp.adam_step([x.copy() for x in params], rW + rb, [z.copy() for z in zeros],
                               [z.copy() for z in zeros], 1, lr=1e-3)
    werr = max(np.max(np.abs(a - r)) for a, r in zip(p_dp, p_1))
    # the replicas hold the same weights after the step
    mine = torch.tensor(np.concatenate([x.reshape(-1) for x in p_dp]))
    other = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(other, mine)
    same = all(torch.equal(other[0], x) for x in other)
    out.put((rank, n, gerr, werr, same))
    dist.destroy_process_group()


def test_two_gloo_ranks_data_parallel_step_equals_single_rank_step():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dp_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, n, gerr, werr, same in res:
        assert n == 2
        assert gerr <= 1e-12, gerr           # mean of the two shares' means = the global mean
        assert werr <= 1e-12, werr
        assert same


def _rebalance_worker(rank, world, port, out):
    """Each rank advanced an equal shard; with the attempt counts it measured, the next step's
    ranges are rebuilt from the whole field's counts."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2312_13513_gb300.parallel import rebalance
    n = 10001
    rng = np.random.default_rng(7)            # the field's per-cell attempt counts (same on all ranks)
    counts = rng.integers(1, 40, n).astype(float)
    counts[: n // 3] *= 5.0                   # a costly flame region at the start of the field
    s, e = shard(n, rank, world)              # first step: equal cell counts
    mine = torch.tensor(counts[s:e] + 1.0)
    ns, ne = rebalance(mine, s, n)
    out.put((rank, s, e, ns, ne))
    dist.destroy_process_group()


def test_rebalance_by_measured_attempts_on_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rebalance_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, s0, e0, a0, b0), (_, s1, e1, a1, b1) = res
    assert s0 == 0 and e0 == s1 and e1 == 10001                     # equal first split
    assert a0 == 0 and b0 == a1 and b1 == 10001                     # new ranges tile the field
    rng = np.random.default_rng(7)
    counts = rng.integers(1, 40, 10001).astype(float)
    counts[: 10001 // 3] *= 5.0
    w = counts + 1.0
    assert b0 < e0                         # the costly first part gets fewer cells
    assert abs(w[:b0].sum() - w[b0:].sum()) <= 2 * w.max()
