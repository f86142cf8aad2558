"""The multi-GPU layout on CPU ranks (gloo, world size 2): disjoint contiguous rollout shares
cover the batch, every served request goes to exactly one rank, the max-over-ranks reduction of
the benchmark, and sharded oracle rollouts gathered on rank 0 equal the unsharded ones."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

from paper_2606_14188_b300 import scenes, shard  # noqa: E402


def test_rollout_range_partitions():
    for total in (0, 1, 7, 1024, 1025):
        for world in (1, 2, 3, 8):
            spans = [shard.rollout_range(total, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == total
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.rollout_range(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import sim as osim
    sc = scenes.rope_scene(8, n_spheres=1, seed=4)
    B, H = 5, 4
    U = scenes.controls_normal_clear(sc, B, H, seed=9)
    osc = osim.Scene(sc["params"], sc["rest_x"])
    lo, hi = shard.rollout_range(B, rank, world)
    mine = np.zeros((B, 3 * 8 + 6))
    for b in range(lo, hi):
        traj, st, _ = osim.rollout(osc, sc["q0"], U[b], "hard")
        mine[b] = traj[-1]
    t = torch.from_numpy(mine)
    dist.all_reduce(t)                               # disjoint shares: the sum is the gather
    slowest = shard.max_over_ranks(1.0 + rank)
    served = [i for i in range(11) if shard.route(i, world) == rank]
    counts = torch.zeros(11, dtype=torch.int64)
    counts[served] = 1
    dist.all_reduce(counts)
    if rank == 0:
        out.put((t.numpy(), slowest, counts.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_cpu_ranks_shard_like_one():
    from oracle import sim as osim
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, slowest, counts = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    sc = scenes.rope_scene(8, n_spheres=1, seed=4)
    U = scenes.controls_normal_clear(sc, 5, 4, seed=9)
    osc = osim.Scene(sc["params"], sc["rest_x"])
    ref = np.stack([osim.rollout(osc, sc["q0"], U[b], "hard")[0][-1] for b in range(5)])
    np.testing.assert_array_equal(gathered, ref)
    assert slowest == 2.0
    assert np.all(counts == 1)
