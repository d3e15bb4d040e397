"""Host-side logic of the multi-rank benchmark path, run as two gloo ranks on
the CPU: the timed region's max over ranks and the whole-job (weak scaling)
MLUPS, and the reference arm's rank filter."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    t = [0.5, 0.8][rank]  # rank 1 is the slow one
    t_max = bench.allreduce_max(t, dist, "cpu")
    q.put((rank, t_max, bench.whole_job_mlups(world, 1000, 10, t_max)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [0.8, 0.8]
    # 2 ranks x 1000 nodes x 10 steps / 0.8 s
    assert all(abs(o[2] - 2 * 1000 * 10 / 0.8 / 1e6) < 1e-12 for o in out)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.allreduce_max(1.25) == 1.25
    assert bench.whole_job_mlups(1, 2_000_000, 5, 0.5) == 20.0


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "3", "--warmup", "3"], env=env, capture_output=True, text=True,
                       timeout=120, cwd=ROOT)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def _sizes():
    sys.path.insert(0, ROOT)
    import synth
    return [s["nx"] * s["ny"] for s in synth.sweep_channels(n=64, seed=3)]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_sweep_shards_partition_the_channels_evenly(world):
    sys.path.insert(0, ROOT)
    from paper_2103_08301_gb300.sweep_bench import shard_channels
    sizes = _sizes()
    shards = shard_channels(sizes, world)
    assert len(shards) == world
    flat = sorted(i for sh in shards for i in sh)
    assert flat == list(range(len(sizes)))  # every channel once
    loads = [sum(sizes[i] for i in sh) for sh in shards]
    assert max(loads) <= 1.05 * sum(sizes) / world
    # largest-first onto the least-loaded rank: no rank could take a channel
    # from the heaviest rank and end lighter than it was
    assert max(loads) - min(loads) <= max(sizes)


def _shard_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2103_08301_gb300.sweep_bench import shard_channels
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    mine = shard_channels(_sizes(), world)[rank]
    got = [None] * world
    dist.all_gather_object(got, mine)
    q.put((rank, got))
    dist.barrier()
    dist.destroy_process_group()


def test_sweep_shards_agree_across_gloo_ranks():
    """Each rank computes its own shard; gathered, the shards are disjoint and
    cover every channel, with no exchange of channel data."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert out[0][1] == out[1][1]
    a, b = out[0][1]
    assert not set(a) & set(b) and sorted(a + b) == list(range(64))
