"""Host-side multi-rank logic of the benchmark with two gloo ranks on CPU:
the path shards macro points across ranks with no collective on the data
path; only the step time is max-reduced and the throughput counts every
rank's points (weak scaling)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    dist.init_process_group('gloo', init_method='tcp://127.0.0.1:%d' % port, rank=rank, world_size=world)
    ms, value = bench.aggregate(1.0 + rank, 1000 * (rank + 1), world, dist, 'cpu')
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_weak_scaling_aggregate_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    # every rank sees the slowest rank's time; throughput = world * local points / max time
    assert out[0][0] == out[1][0] == 2.0
    assert out[0][1] == pytest.approx(world * 1000 / 2e-3)
    assert out[1][1] == pytest.approx(world * 2000 / 2e-3)


def test_reference_arm_other_ranks_exit_quietly():
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK='1', WORLD_SIZE='2', LOCAL_RANK='1')
    r = subprocess.run([sys.executable, os.path.join(root, 'bench.py'), '--impl', 'reference', '--steps', '1',
                        '--warmup', '0'], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ''
