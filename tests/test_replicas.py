"""bench.py --gpus N runs N independent replicas (the single-LP path does not
shard): the whole-job rate is the iterations of all ranks over the slowest
rank's time.  Checked with two gloo ranks on the CPU."""
import os
import socket
import subprocess
import sys

from conftest import ROOT

CHILD = r"""
import os, sys
sys.path.insert(0, %r)
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
elapsed = [2.0, 5.0][rank]  # the second replica is slower
value, emax = bench.replica_rate(elapsed, steps=10, world=world)
assert emax == 5.0 and abs(value - 10 * 2 / 5.0) < 1e-12, (value, emax)
w, r, l = bench.dist_info()
assert (w, r) == (world, rank)
dist.barrier()
dist.destroy_process_group()
print("rank", rank, "ok", value)
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_replicas_take_the_max_time():
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                   LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD % ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (out, err) in zip(procs, outs):
        assert p.returncode == 0, err
        assert "ok" in out


def test_single_process_rate():
    sys.path.insert(0, ROOT)
    import bench
    value, emax = bench.replica_rate(4.0, steps=8, world=1)
    assert value == 2.0 and emax == 4.0
