"""Multi-process path on the CPU: two gloo ranks run the replica helpers the benchmark
uses for N > 1 (barrier, max and sum over ranks, the whole-job rate) and the
partition of independent graphs among ranks."""
import json
import os
import socket
import subprocess
import sys

import pytest

from paper_2303_03964_gb300 import replicas

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, sys
import torch.distributed as dist
from paper_2303_03964_gb300 import replicas
ws, rank, local = replicas.world()
dist.init_process_group("gloo", timeout=__import__("datetime").timedelta(seconds=60))
replicas.barrier()
secs = [2.0, 3.5][rank]           # rank 1 is the slow one
units = [1000, 1000][rank]
out = {"rank": rank, "ws": ws, "max": replicas.max_over_ranks(secs),
       "sum": replicas.sum_over_ranks(units), "rate": replicas.throughput(units, secs),
       "shard": list(replicas.shard(512, rank, ws))}
replicas.barrier()
dist.destroy_process_group()
print(json.dumps(out))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), PYTHONPATH=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            so, se = p.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        assert p.returncode == 0, se
        outs.append(json.loads(so.strip().splitlines()[-1]))
    for o in outs:
        assert o["ws"] == 2
        assert o["max"] == 3.5          # the slowest rank's time
        assert o["sum"] == 2000.0       # units of both ranks
        assert o["rate"] == pytest.approx(2000.0 / 3.5)
    # the two shares partition the 512 graphs
    shards = [o["shard"] for o in sorted(outs, key=lambda o: o["rank"])]
    assert shards[0] + shards[1] == list(range(512))


def test_single_process_fallbacks():
    assert replicas.max_over_ranks(1.5) == 1.5
    assert replicas.sum_over_ranks(7) == 7.0
    assert replicas.throughput(10, 2.0) == 5.0
    replicas.barrier()


@pytest.mark.parametrize("count,ws", [(0, 1), (1, 4), (512, 3), (7, 7), (1000, 8)])
def test_shard_partitions(count, ws):
    parts = [list(replicas.shard(count, r, ws)) for r in range(ws)]
    assert sum(parts, []) == list(range(count))
    sizes = [len(p) for p in parts]
    assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.shard(count, ws, ws)
