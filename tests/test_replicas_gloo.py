"""The N > 1 path of bench.py on the CPU: replicas are independent, so the only cross-rank
steps are the barrier and the max over ranks of the timings, which two gloo processes
exercise here (no GPU).  Also: under torchrun the reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dev_s, wall = bench.reduce_max([times[rank], 10.0 * times[rank]], dist)
        dist.barrier()
        out.put((rank, dev_s, wall, bench.replica_value(3.0e12, 5, world, dev_s)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [2.0, 3.0]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, dev_s, wall, value in res:
        assert dev_s == 3.0 and wall == 30.0          # the slowest rank sets the time
        assert value == pytest.approx(3.0e12 * 5 * 2 / 3.0 / 1e12)


def test_single_process_reduce_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max([1.5, 2.5]) == [1.5, 2.5]
    assert bench.replica_value(2.0e12, 4, 1, 2.0) == pytest.approx(4.0)


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0", "--n", "256", "--b", "16", "--ref-panels", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env = dict(os.environ, RANK="0", WORLD_SIZE="2", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0", "--n", "256", "--b", "16", "--ref-panels", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_partition_systems_is_flop_balanced():
    """Independent systems (batched and served forms) split over GPUs: every system in
    exactly one part, and the largest part within one system's work of the average (the
    largest-first greedy rule)."""
    sys.path.insert(0, ROOT)
    import prrp_inputs as pi
    from paper_1208_2451_gb300 import binding as B
    sizes = [int(k) for k in pi.batch_sizes(4096, 32, 512, 0)]
    for parts in (1, 2, 3, 4, 8):
        split = B.partition_systems(sizes, parts)
        flat = sorted(i for p in split for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] ** 3 for i in p) for p in split]
        assert max(loads) <= sum(loads) / parts + max(s ** 3 for s in sizes)
    assert B.partition_systems([5, 5, 5], 2) == [[0, 2], [1]]


def _shard_worker(rank, world, port, sizes, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1208_2451_gb300 import binding as B
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = B.partition_systems(sizes, world)[rank]
        everyone = [None] * world
        dist.all_gather_object(everyone, mine)          # host-side gather of the shards
        out.put((rank, everyone))
    finally:
        dist.destroy_process_group()


def test_sharded_batch_covers_every_system_once():
    import torch.multiprocessing as mp
    pytest.importorskip("paper_1208_2451_gb300.binding", reason="libprrp.so not built")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    sizes = [37, 512, 64, 300, 129, 480, 33, 256, 200, 511]
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for _, everyone in res:
        flat = sorted(i for part in everyone for i in part)
        assert flat == list(range(len(sizes)))
        assert everyone == res[0][1]                    # every rank agrees on the split
