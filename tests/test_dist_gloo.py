"""The multi-rank path of bench.py on CPU: two gloo ranks (127.0.0.1), each
with its own replica time; the job time is the maximum over ranks and the
rate counts every rank's units.  The batched ensemble is sharded by member:
the ranks' shares are disjoint, cover every member once and balance the node
count; the job's node updates are the sum over ranks.  The reference arm
prints only on rank 0."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(10.0 + 5.0 * rank, world)
    rate = bench.whole_job_rate(100.0, world, t)
    units = bench.sum_over_ranks(100.0 + 50.0 * rank, world)
    out.put((rank, t, rate, units))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 15.0, 200.0 / 15.0, 250.0), (1, 15.0, 200.0 / 15.0, 250.0)]


def test_ensemble_members_are_sharded_disjointly():
    sys.path.insert(0, ROOT)
    import bench

    class M:          # stands in for inputs.EnsembleMember: only identity and size matter here
        def __init__(self, r, n):
            self.r, self.n = r, n

    rng = __import__("numpy").random.default_rng(0)
    every = [M(r, int(n)) for r, n in enumerate(rng.choice([2400, 9500, 38400, 152000], 256))]
    for world in (1, 2, 4, 8):
        shares = [bench.shard_members(every, rank, world) for rank in range(world)]
        ids = sorted(m.r for sh in shares for m in sh)
        assert ids == list(range(256))
        sizes = [sum(m.n for m in sh) for sh in shares]
        assert max(sizes) < 1.35 * (sum(sizes) / world), (world, sizes)


def test_reference_arm_prints_only_on_rank_zero():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
