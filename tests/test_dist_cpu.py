"""The multi-process side of bench.py on CPU: two gloo ranks exchange their
timings (max over ranks) and pass the barrier, as the torchrun launch of
bench.py does with one GPU per rank (products are independent per rank, so
no data-path collective exists)."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys
sys.path.insert(0, %r)
import bench
world, rank, local = bench.dist_env()
dist = bench.dist_init(world, "gloo")
bench.barrier(dist)
mine = 1.5 if rank == 0 else 4.25
most = bench.max_over_ranks(dist, mine)
assert most == 4.25, most
bench.barrier(dist)
dist.destroy_process_group()
print("rank", rank, "ok", most)
""" % ROOT


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_gloo_ranks_max_and_barrier():
    pytest.importorskip("torch.distributed")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
    outs = []
    for p in procs:
        out, _ = p.communicate(timeout=120)
        outs.append(out.decode())
        assert p.returncode == 0, out.decode()
    assert all("ok 4.25" in o for o in outs)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_init(1, "gloo") is None
    assert bench.max_over_ranks(None, 3.0) == 3.0


SHARD_CHILD = r"""
import os, sys
sys.path.insert(0, %r)
import bench
import workloads as W
from paper_1612_05778_gb300 import shard
world, rank, local = bench.dist_env()
dist = bench.dist_init(world, "gloo")
shapes = W.batch_shapes(seed=3, count=4096)
costs = shard.shape_costs([(s.na, s.nb, s.bits_a, s.bits_b) for s in shapes])
mine = shard.partition(costs, world)[rank]
got = [None] * world
dist.all_gather_object(got, mine)
flat = sorted(i for part in got for i in part)
assert flat == list(range(len(shapes))), "every product exactly once"
ld = [sum(costs[i] for i in part) for part in got]
assert max(ld) - min(ld) <= max(costs), ld
mine_load = sum(costs[i] for i in mine)
assert bench.max_over_ranks(dist, mine_load) == max(ld)
dist.destroy_process_group()
print("rank", rank, "shard ok", len(mine))
""" % ROOT


def test_two_gloo_ranks_split_the_batch():
    """The batched workload under torchrun: each rank computes the same
    cost-balanced split of the 4096 products (no message needed to agree);
    gathered over gloo, every product is assigned exactly once and the
    loads differ by at most one product's cost."""
    pytest.importorskip("torch.distributed")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", SHARD_CHILD], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
    for p in procs:
        out, _ = p.communicate(timeout=300)
        assert p.returncode == 0, out.decode()
        assert "shard ok 2048" in out.decode()


def test_partition_bounds_on_skewed_costs():
    from paper_1612_05778_gb300 import shard
    costs = [1000.0] + [1.0] * 50 + [37.5, 12.0, 999.0]
    for world in (1, 2, 3, 8):
        parts = shard.partition(costs, world)
        assert sorted(i for p in parts for i in p) == list(range(len(costs)))
        ld = shard.loads(costs, parts)
        assert max(ld) - min(ld) <= max(costs)
    assert shard.partition([], 4) == [[], [], [], []]
