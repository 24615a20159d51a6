"""Host-side multi-rank logic with two gloo ranks on CPU.  The benchmark
shards macro points across ranks with no collective on the data path; only
the step time is max-reduced and the throughput counts every rank's points
(weak scaling).  A monolithic Newton iteration shards the macro mesh by
element range; the ranks' partial systems are summed by one all-reduce."""
import os
import socket

import pytest
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
    mgr = mp.get_context('spawn').Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    # every rank sees the slowest rank's time; throughput = world * local points / max time
    assert out[0][0] == out[1][0] == 2.0
    assert out[0][1] == pytest.approx(world * 1000 / 2e-3)
    assert out[1][1] == pytest.approx(world * 2000 / 2e-3)


def test_element_ranges_partition_the_mesh():
    from paper_2306_02687_gb300.parallel import element_range
    for n_elem in (0, 1, 5, 64, 1001):
        for world in (1, 2, 3, 8):
            rs = [element_range(n_elem, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n_elem
            assert all(rs[k][1] == rs[k + 1][0] for k in range(world - 1))
            sizes = [b - a for a, b in rs]
            assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        element_range(10, 2, 2)


def _shard_worker(rank, world, port, out):
    # every rank assembles its element range with the float64 oracle (the
    # other ranges' points contribute nothing), the partial systems are
    # summed through the package's all-reduce, and so are the norms
    import numpy as np
    import torch
    import synthetic as syn
    from synthetic import meshes
    from oracle import macro
    from paper_2306_02687_gb300 import parallel
    dist.init_process_group('gloo', init_method='tcp://127.0.0.1:%d' % port, rank=rank, world_size=world)
    X, conn = meshes.rect(5, 3, 1.5, 1.0)
    om = macro.MacroMesh(X, conn)
    P = syn.perturbation(syn.SEED_BASE + 70, (om.n_ip, 2, 2), 0.1)
    C = syn.perturbation(syn.SEED_BASE + 71, (om.n_ip, 4, 4), 1.0)
    e0, e1 = parallel.element_range(om.n_el, rank, world)
    keep = np.zeros(om.n_ip, dtype=bool)
    keep[e0 * om.ngp:e1 * om.ngp] = True
    R, K = om.assemble(np.where(keep[:, None, None], P, 0.0), np.where(keep[:, None, None], C, 0.0))
    buf = torch.from_numpy(np.concatenate([R, K.toarray().ravel()]))
    parallel.allreduce_system(buf)
    norms = torch.tensor([1.0, 2.0, 0.5 + rank], dtype=torch.float64)
    parallel.allreduce_norms(norms)
    Rf, Kf = om.assemble(P, C)
    full = np.concatenate([Rf, Kf.toarray().ravel()])
    out[rank] = (float(np.abs(buf.numpy() - full).max() / np.abs(full).max()), norms.tolist(), e1 - e0)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_assembly_all_reduce_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context('spawn').Manager()
    out = mgr.dict()
    mp.spawn(_shard_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        err, norms, n_el = out[r]
        assert err <= 1e-14
        assert norms == [1.0, 2.0, 1.5]
        assert n_el == 8 if r == 0 else n_el == 7


def test_reference_arm_other_ranks_exit_quietly():
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK='1', WORLD_SIZE='2', LOCAL_RANK='1')
    r = subprocess.run([sys.executable, os.path.join(root, 'bench.py'), '--impl', 'reference', '--steps', '1',
                        '--warmup', '0'], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ''


def test_reference_arm_json_line():
    # rank 0 of the reference arm prints one JSON line with the contract's keys
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ('RANK', 'WORLD_SIZE', 'LOCAL_RANK')}
    r = subprocess.run([sys.executable, os.path.join(root, 'bench.py'), '--impl', 'reference', '--steps', '1',
                        '--warmup', '1'], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ('metric', 'value', 'unit', 'n_gpus', 'steps', 'warmup', 'ms_per_step', 'higher_is_better',
                'scaling', 'vs_baseline', 'dtype', 'data', 'config', 'cpu_baseline', 'e2e'):
        assert key in d, key
    assert d['impl'] == 'reference' and d['n_gpus'] == 1 and d['steps'] == 1 and d['warmup'] == 1
    assert d['value'] > 0 and d['higher_is_better'] is True and d['unit'] == 'RVE evals/s'
    assert d['ms_per_step'] > 0 and 'workload' in d['config']
    assert d['cpu_baseline']['kind'] == 'oracle' and d['cpu_baseline']['cores'] >= 1
    assert d['cpu_baseline']['value'] == d['value'] and isinstance(d['cpu_baseline']['sample'], str)
    assert d['e2e']['value'] == d['value'] and d['e2e']['unit'] == d['unit']
    assert d['e2e']['h2d_bytes_per_step'] == 0 and d['e2e']['d2h_bytes_per_step'] == 0
