"""Throughput of the hyper-ROM FE^2 online step on GB300.

A step is one monolithic Newton iteration of the hot path over a fixed
synthetic batch: macro deformation gradient at every macro Gauss point ->
batched hyper-reduced RVE evaluation (polar split, micro update, ECM loop,
static condensation, rotation back) -> macro element assembly of R and K ->
convergence scalars.  The metric is RVE evaluations per second (one
evaluation = one macro point in one Newton iteration).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c1..c5]
                  [--precision mixed|fp64] [--impl ours|reference]
                  [--candidate I] [--no-cpu-baseline] [--no-oracle-check]

--candidate pins one compiled kernel configuration instead of the
autotuner's pick (as named by rve_rom_kernel_info); --no-cpu-baseline skips
the timed oracle sample; --no-oracle-check skips the accuracy check of the
timed form against the float64 oracle on 256 sampled points (mid-Newton
states the oracle converged), reported per output in accuracy_vs_oracle.

Default workload c2: 2D plane strain, 48x48 Q4 RVE with 4 inclusions, 24
modes, 200 ECM points, plate with a central hole (O-grid 4 x 32 x 32 Q4,
16384 macro Gauss points).  The CPU baseline and the reference arm time the
float64 oracle as it stands on a bounded sample of the same points.
"""
import os

for _v in ('OMP_NUM_THREADS', 'OPENBLAS_NUM_THREADS', 'MKL_NUM_THREADS'):
    os.environ.setdefault(_v, '1')

import argparse  # noqa: E402
import json  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import tempfile  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as syn  # noqa: E402
from synthetic import meshes  # noqa: E402

METRIC = "hyper-ROM RVE evals/s on 1 GB300, batched FP32/FP64 vs plain FP64, P̄ err ≤1e-8"
UNIT = "RVE evals/s"

WORKLOADS = {
    'c1': dict(roms=['c1'], d=2, mesh=('rect', (4, 4)), load=0.10, desc='2D 16x16 Q4 RVE, 12 modes, 60 ECM points, 4x4 Q4 macro (64 points)'),
    'c2': dict(roms=['c2'], d=2, mesh=('plate', (32, 32)), load=0.15,
               desc='2D 48x48 Q4 RVE (4 inclusions), 24 modes, 200 ECM points, plate with hole 4x32x32 Q4 (16384 points)'),
    'c3': dict(roms=['c3'], d=3, mesh=('box', (32, 32, 8, 4.0, 4.0, 1.0)), load=0.20,
               desc='3D 16^3 hex8 RVE, 40 modes, 400 ECM points, 32x32x8 hex8 cantilever (65536 points)'),
    'c4': dict(roms=['c1'], d=2, mesh=('rect', (64, 64)), load=0.10,
               desc='2D 16x16 Q4 RVE, 12 modes, 60 ECM points, 64x64 Q4 macro (16384 points)'),
    'c5': dict(roms=['c5a', 'c5b', 'c5c'], d=2, mesh=('rect', (181, 181)), load=0.14,
               desc='2D mixed batch of 3 RVE types (16/32/64 modes, 120/300/600 ECM points), 181x181 Q4 (131044 points)'),
}

# DRAM traffic per launch of the evaluation kernel from one ncu capture of
# this workload (the warp-specialized tensor-core kernel the autotuner picks
# for the mixed form, and the float64 kernel); reported only for that
# workload and form, and to be refreshed whenever the kernel changes.
PROFILED_TRAFFIC = {('c2', 'mixed'): 17201408, ('c2', 'fp64'): 17142784}

# algorithmic work per evaluation (FP64 FLOP of kinematics + residual + law,
# symmetric-half tangent contraction FLOP), per ROM type
def work_per_eval(rom):
    m, g, n = rom['B'].shape
    d = int(round(np.sqrt(g)))
    law = 150 if d == 2 else 400
    fp64 = 2 * m * g * n * 2 + m * (law + 2 * g)
    fp32 = n * (n + 1) * m * g + 2 * m * g * g * n
    return fp64, fp32


def macro_displacement(X, load, seed):
    """Smooth synthetic macro displacement: uniform stretch `load/2` plus
    seeded sine modes with displacement gradients of about load/3."""
    g = syn.rng(seed)
    d = X.shape[1]
    L = X.max(0) - X.min(0)
    u = 0.5 * load * X.copy()
    for k in range(1, 4):
        for i in range(d):
            ph = g.random(d) * 2 * np.pi
            amp = (load / 3.0) * (g.random() - 0.5) / (k * np.pi) * L.min()
            arg = sum(2 * np.pi * k * X[:, j] / L[j] + ph[j] for j in range(d))
            u[:, i] += amp * np.sin(arg)
    return u


def build_mesh(spec):
    kind, a = spec
    if kind == 'rect':
        return meshes.rect(*a)
    if kind == 'box':
        return meshes.box(*a)
    return meshes.plate_with_hole(*a)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix='.csv')
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ['nvidia-smi', '-i', str(self.index),
                 '--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,'
                 'clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,'
                 'clocks_event_reasons.sw_power_cap', '--format=csv,noheader,nounits', '-lms', '200'],
                stdout=open(self.path, 'w'), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(',')]
                if len(f) < 6:
                    continue
                try:
                    sm.append(float(f[0]))
                    mx.append(float(f[1]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[2:6]):
                    if v.lower().startswith('active'):
                        reasons.add(nm)
            os.unlink(self.path)
        except Exception:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate(ms_local, n_local, world, dist=None, device='cpu'):
    """Weak-scaling aggregate over ranks: the step time is the maximum over
    ranks and the throughput counts the points of every rank.  Returns
    (ms_max, whole-job evaluations per second)."""
    ms = float(ms_local)
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * n_local / (ms * 1e-3)


def host_cores():
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    try:
        out = subprocess.run(['lscpu'], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith('Model name:'):
                return line.split(':', 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open('/proc/cpuinfo'):
            if line.lower().startswith('model name'):
                return line.split(':', 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


_WORKER = {}


def _oracle_worker_init(rom_paths):
    from oracle import reduced
    _WORKER['roms'] = [reduced.Rom.load(p) for p in rom_paths]


def _oracle_worker_run(job):
    """Evaluate the points of one chunk with the float64 oracle (fresh state
    at each point's Fbar): once through the chunk (budget None), or cycling
    until `budget` seconds have passed.  Returns (evaluations, seconds)."""
    from oracle import polar, reduced, rve
    types, F, budget = job
    roms = _WORKER['roms']
    states = []
    for a in range(len(F)):
        st = reduced.zero_state(roms[types[a]])
        st['Uprev'] = rve.to_voigt(polar.polar(F[a])[1])
        states.append(st)
    cnt, a = 0, 0
    t0 = time.perf_counter()
    while True:
        reduced.eval_point(roms[types[a]], F[a], **states[a])
        cnt += 1
        a = (a + 1) % len(F)
        el = time.perf_counter() - t0
        if (budget is None and cnt == len(F)) or (budget is not None and el >= budget):
            return cnt, el


class OraclePool:
    """The float64 oracle as it stands, one process per host core (spawned
    processes, one NumPy thread each)."""

    def __init__(self, rom_paths, cores):
        import multiprocessing
        self.cores = cores
        self.pool = multiprocessing.get_context('spawn').Pool(cores, initializer=_oracle_worker_init,
                                                              initargs=(rom_paths,))

    def chunks(self, types, F, budget):
        k = self.cores
        return [(types[i::k], F[i::k], budget) for i in range(k) if len(F[i::k])]

    def run(self, types, F, budget=None):
        return self.pool.map(_oracle_worker_run, self.chunks(types, F, budget), chunksize=1)

    def close(self):
        self.pool.close()
        self.pool.join()


def native_cpu_rate(rom_list, types_np, F, sel_all, nthreads, target_s=1.0, runs=5):
    """Median of `runs` timings (evaluations/s) of the plain C++ float64
    baseline on `nthreads` threads over a sample of the workload's points
    sized to take about target_s seconds per run (fresh states).  Returns
    (rate, threads used, points per run)."""
    import cpu_baseline

    def one(sel):
        t0 = time.perf_counter()
        used = 1
        for t, rom in enumerate(rom_list):
            idx = sel[types_np[sel] == t]
            if len(idx) == 0:
                continue
            m, g, nm = rom['B'].shape
            d = int(round(np.sqrt(g)))
            ns = 3 if d == 2 else 6
            q = np.zeros((len(idx), nm))
            s_ = np.zeros((len(idx), nm))
            S_ = np.zeros((len(idx), nm, ns))
            U_ = np.zeros((len(idx), ns))
            U_[:, :d] = 1.0
            _, used = cpu_baseline.eval_batch(rom, F[idx], q, s_, S_, U_, nthreads=nthreads)
        return time.perf_counter() - t0, used
    probe = sel_all[:max(8, 2 * nthreads)]
    dt, _ = one(probe)
    per_pt = dt / len(probe)
    npts = int(min(len(sel_all), max(len(probe), target_s / max(per_pt, 1e-9))))
    sel = sel_all[:npts]
    times, used = [], 1
    for _ in range(runs):
        dt, used = one(sel)
        times.append(dt)
    return npts / statistics.median(times), used, npts


def oracle_accuracy(rom_paths, types_np, F_or, sel, seed):
    """Oracle inputs and outputs at the sampled points: a mid-Newton state per
    point (micro state converged by the oracle at a nearby Fbar, the stored
    s, S, U_prev of that evaluation, q perturbed by 1e-3 of its size), then
    one oracle evaluation at the workload's Fbar.  Inputs come from the
    oracle and the seeded generators only."""
    from oracle import reduced
    roms = [reduced.Rom.load(p) for p in rom_paths]
    states, outs = [], []
    for k, a in enumerate(sel):
        r = roms[types_np[a]]
        F1 = F_or[a]
        F0 = F1 - syn.perturbation(seed + 2 * k, F1.shape, 2e-3)
        o, _ = reduced.converge_point(r, F0)
        q = o['q'] + syn.perturbation(seed + 2 * k + 1, r.n, 1e-3 * np.abs(o['q']).max())
        st = dict(q=q, s=o['s'], S=o['S'], Uprev=o['Uprev'])
        states.append(st)
        outs.append(reduced.eval_point(r, F1, **st))
    return states, outs


def accuracy_report(g, outs, sel, types_np, rom_n):
    """Largest relative error per output over the sampled points (P, dPdF
    relative to the point's largest entry; s, S, q likewise; rnorm relative
    to itself)."""
    def rel(x, y):
        return float(np.abs(x - y).max() / max(np.abs(y).max(), 1e-300))
    errs = dict(Pbar=0.0, dPdF=0.0, s=0.0, S=0.0, q=0.0, rnorm=0.0)
    bad = 0
    for k, (a, o) in enumerate(zip(sel, outs)):
        if g['status'][k] != 0 or o['status'] != 0:
            bad += 1
            continue
        n = rom_n[types_np[a]]
        errs['Pbar'] = max(errs['Pbar'], rel(g['Pbar'][k], o['Pbar'].ravel()))
        errs['dPdF'] = max(errs['dPdF'], rel(g['dPdF'][k], o['dPdF']))
        errs['s'] = max(errs['s'], rel(g['s'][k][:n], o['s']))
        errs['S'] = max(errs['S'], rel(g['S'][k][:n], o['S']))
        errs['q'] = max(errs['q'], rel(g['q'][k][:n], o['q']))
        errs['rnorm'] = max(errs['rnorm'], abs(g['rnorm'][k] - o['rnorm']) / max(o['rnorm'], 1e-300))
    out = {k + '_rel_err_max': v for k, v in errs.items()}
    out['points'] = len(sel)
    out['failed_points'] = bad
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=10)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--workload', default='c2', choices=sorted(WORKLOADS))
    ap.add_argument('--precision', default='mixed', choices=['mixed', 'fp64'])
    ap.add_argument('--impl', default='ours', choices=['ours', 'reference'])
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--no-adjoint', action='store_true', help='skip the timing of the implicit adjoint')
    ap.add_argument('--no-other-workloads', action='store_true',
                    help='skip the evaluation throughput of the other workloads (c1, c3, c4, c5)')
    ap.add_argument('--no-newton', action='store_true',
                    help='skip the timing of whole Newton iterations with the global macro solve')
    ap.add_argument('--no-oracle-check', action='store_true',
                    help='skip the per-output comparison with the float64 oracle on 256 sampled points')
    ap.add_argument('--candidate', type=int, default=-1,
                    help='force this forward kernel candidate (rve_rom_select_kernel) for every type and '
                         'precision after autotuning; -1 keeps the autotuner\'s choice')
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    rank = int(os.environ.get('RANK', '0'))
    world = int(os.environ.get('WORLD_SIZE', '1'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    rom_paths = [os.path.join(ROOT, 'tests', 'golden', 'rom_%s.npz' % r) for r in wl['roms']]

    X, conn = build_mesh(wl['mesh'])
    d = wl['d']
    u_host = macro_displacement(X, wl['load'], syn.SEED_BASE + 500 + rank)

    if args.impl == 'reference':
        if rank != 0:
            return 0
        run_reference(args, wl, rom_paths, X, conn, u_host)
        return 0

    import torch
    import paper_2306_02687_gb300 as rv

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl')
    dev = torch.device('cuda', local)

    roms = [rv.load_rom_file(p) for p in rom_paths]
    h = rv.rve_rom_create(d, roms, roms[0]['V0'])
    tune = {prec: rv.rve_rom_autotune(h, prec, n_sample=16384).round(4).tolist() for prec in ('mixed', 'fp64')}
    if args.candidate >= 0:
        for prec in ('mixed', 'fp64'):
            for t in range(len(roms)):
                nc = rv.rve_rom_select_kernel(h, t, prec)
                rv.rve_rom_select_kernel(h, t, prec, min(args.candidate, nc - 1))
    mesh = rv.macro_mesh_create(X, conn)
    n = mesh.n_ip
    types = None
    types_np = np.zeros(n, dtype=np.int32)
    if len(roms) > 1:
        types_np = syn.type_labels(syn.SEED_BASE + 600 + rank, n, len(roms))
        types = torch.tensor(types_np, device=dev)
    u = torch.tensor(u_host, device=dev)
    Fbar = torch.empty(n, d * d, dtype=torch.float64, device=dev)
    rv.macro_gradient(mesh, u, Fbar)
    q, s, S, U = h.zero_state(n)
    Pbar, dPdF, rnorm, status = h.outputs(n)
    R = torch.empty(mesh.n_dof, dtype=torch.float64, device=dev)
    Kv = torch.empty(mesh.nnz, dtype=torch.float64, device=dev)
    free = torch.ones(mesh.n_dof, dtype=torch.uint8, device=dev)
    norms = torch.empty(3, dtype=torch.float64, device=dev)

    # mid-Newton state: micro states converged at Fbar (float64 staggered
    # iterations), then q perturbed by 1e-3 of its size
    for _ in range(8):
        rv.rve_rom_eval_batch(h, Fbar, q, s, S, U, Pbar, dPdF, rnorm, status, type=types, precision='fp64')
    g = torch.Generator(device='cpu').manual_seed(syn.SEED_BASE + 700 + rank)
    pert = torch.randn(q.shape, generator=g, dtype=torch.float64).to(dev)
    q += 1e-3 * q.abs().amax(dim=1, keepdim=True) * pert * (q != 0)
    s.zero_()
    S.zero_()
    torch.cuda.synchronize()
    bad = int((status != 0).sum().item())
    state0 = [x.clone() for x in (q, s, S, U)]

    def restore():
        for x, y in zip((q, s, S, U), state0):
            x.copy_(y)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(precision, ev=None):
        rv.macro_gradient(mesh, u, Fbar)
        if ev is not None:
            ev[0].record(stream)
        rv.rve_rom_eval_batch(h, Fbar, q, s, S, U, Pbar, dPdF, rnorm, status, type=types, precision=precision)
        if ev is not None:
            ev[1].record(stream)
        rv.macro_assemble(mesh, Pbar, dPdF, R, Kv)
        rv.macro_residual_norms(mesh, R, free, rnorm, norms)

    def timed(precision, steps, warmup):
        restore()
        for _ in range(warmup):
            step(precision)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        tot, kern = 0.0, 0.0
        for _ in range(steps):
            flush.zero_()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            e[0].record(stream)
            step(precision, (e[1], e[2]))
            e[3].record(stream)
            e[3].synchronize()
            tot += e[0].elapsed_time(e[3])
            kern += e[1].elapsed_time(e[2])
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        return tot / steps, kern / steps

    with ClockSampler(local) as clk:
        ms_step, ms_kern = timed(args.precision, args.steps, args.warmup)
    clocks = clk.summary()
    ms_max, value = aggregate(ms_step, n, world, dist, dev)

    # plain float64 GPU form on the same workload (speedup denominator)
    other = 'fp64' if args.precision == 'mixed' else 'mixed'
    ms_other, _ = timed(other, max(2, min(args.steps, 5)), 1)

    # accuracy of the timed form against the float64 form on every point
    restore()
    rv.rve_rom_eval_batch(h, Fbar, q, s, S, U, Pbar, dPdF, rnorm, status, type=types, precision=args.precision)
    P1, C1 = Pbar.clone(), dPdF.clone()
    restore()
    rv.rve_rom_eval_batch(h, Fbar, q, s, S, U, Pbar, dPdF, rnorm, status, type=types, precision='fp64')
    torch.cuda.synchronize()
    pn = Pbar.abs().amax(dim=1).clamp_min(1e-300)
    cn = dPdF.abs().amax(dim=(1, 2)).clamp_min(1e-300)
    p_pt = (P1 - Pbar).abs().amax(dim=1) / pn
    p_err = p_pt.max().item()
    c_err = ((C1 - dPdF).abs().amax(dim=(1, 2)) / cn).max().item()
    p_err_type = None
    if types is not None:      # per RVE type of a mixed batch
        p_err_type = {wl['roms'][t]: float(p_pt[types == t].max().item()) for t in range(len(roms))}

    # accuracy of the timed form against the float64 oracle, per output, on
    # 256 sampled points that carry oracle mid-Newton states (the workload's
    # Fbar from the oracle's macro gradient of the same displacement field)
    acc = None
    if not args.no_oracle_check:
        from oracle import macro as omacro
        F_or = omacro.MacroMesh(X, conn).gradient(u_host)
        sel = np.sort(syn.rng(syn.SEED_BASE + 800 + rank).choice(n, min(n, 256), replace=False))
        states, outs = oracle_accuracy(rom_paths, types_np, F_or, sel, syn.SEED_BASE + 900 + 1000 * rank)
        restore()
        si = torch.tensor(sel, device=dev)
        Fbar[si] = torch.tensor(F_or[sel].reshape(len(sel), d * d), device=dev)
        for k, st in enumerate(states):
            nk = len(st['q'])
            for x, v in ((q, st['q']), (s, st['s']), (S, st['S'])):
                x[sel[k]].zero_()
                x[sel[k], :nk] = torch.tensor(v, device=dev)
            U[sel[k]] = torch.tensor(st['Uprev'], device=dev)
        rv.rve_rom_eval_batch(h, Fbar, q, s, S, U, Pbar, dPdF, rnorm, status, type=types,
                              precision=args.precision)
        torch.cuda.synchronize()
        g_acc = {k: v[si].cpu().numpy() for k, v in dict(Pbar=Pbar, dPdF=dPdF, s=s, S=S, q=q, rnorm=rnorm,
                                                          status=status).items()}
        acc = accuracy_report(g_acc, outs, sel, types_np, [r['B'].shape[2] for r in roms])
        acc["gate"] = {"Pbar": 1e-8, "dPdF": 1e-5}
        acc["meets_gate"] = bool(acc['failed_points'] == 0 and acc['Pbar_rel_err_max'] <= 1e-8
                                 and acc['dPdF_rel_err_max'] <= 1e-5)

    # end to end through the public API: pinned host u in, R / K / norms out
    u_pin = torch.tensor(u_host).pin_memory()
    R_pin = torch.empty(mesh.n_dof, dtype=torch.float64).pin_memory()
    K_pin = torch.empty(mesh.nnz, dtype=torch.float64).pin_memory()
    nrm_pin = torch.empty(3, dtype=torch.float64).pin_memory()
    restore()
    e2e_steps = max(2, min(args.steps, 10))
    for it in range(1 + e2e_steps):
        if it == 1:
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        u.copy_(u_pin, non_blocking=True)
        step(args.precision)
        R_pin.copy_(R, non_blocking=True)
        K_pin.copy_(Kv, non_blocking=True)
        nrm_pin.copy_(norms, non_blocking=True)
    e1.record(stream)
    e1.synchronize()
    ms_e2e, e2e_value = aggregate(e0.elapsed_time(e1) / e2e_steps, n, world, dist, dev)

    # the same step captured once in a CUDA graph and replayed
    restore()
    step(args.precision)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph):
            step(args.precision)
    restore()
    torch.cuda.synchronize()
    gms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        graph.replay()
        g1.record(stream)
        g1.synchronize()
        gms += g0.elapsed_time(g1)
    ms_graph, graph_value = aggregate(gms / args.steps, n, world, dist, dev)

    # a whole monolithic Newton iteration on the device: the step above plus
    # the global macro solve (macro_solve) and the update u += du, with the
    # workload's boundary DOFs held at the synthetic field's values
    # the implicit adjoint (rve_rom_adjoint) over every point at converged
    # micro states: a cotangent on Pbar -> cotangents on Fbar and the moduli
    adj = None
    if not args.no_adjoint:
        restore()
        for _ in range(12):
            rv.rve_rom_eval_batch(h, Fbar, q, s, S, U, Pbar, dPdF, rnorm, status, type=types, precision='fp64')
        gP = torch.randn(n, d * d, dtype=torch.float64, device=dev,
                         generator=torch.Generator(device=dev).manual_seed(syn.SEED_BASE + 710))
        gF = torch.empty_like(gP)
        gth = torch.zeros(len(roms), 2, 2, dtype=torch.float64, device=dev)
        ast = torch.empty(n, dtype=torch.int32, device=dev)
        for _ in range(args.warmup):
            rv.rve_rom_adjoint(h, Fbar, q, gP, gF, gth, ast, type=types)
        torch.cuda.synchronize()
        ams = 0.0
        for _ in range(args.steps):
            flush.zero_()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            rv.rve_rom_adjoint(h, Fbar, q, gP, gF, gth, ast, type=types)
            a1.record(stream)
            a1.synchronize()
            ams += a0.elapsed_time(a1)
        ams /= args.steps
        adj = {"value": n / (ams * 1e-3), "unit": "adjoint point evaluations/s", "ms_per_call": ams, "points": n,
               "converged_rnorm_max": rnorm.max().item(), "failed_points": int((ast != 0).sum().item()),
               "note": "rve_rom_adjoint (float64) at micro states converged by 12 float64 evaluations"}
        restore()

    others = None
    if not args.no_other_workloads and world == 1:
        others = other_workloads(rv, [w for w in ('c1', 'c3', 'c4', 'c5') if w != args.workload],
                                 args.precision, max(3, min(args.steps, 5)), dev, flush)

    newton = None
    if not args.no_newton:
        newton = newton_leg(rv, h, mesh, wl, u_host, Fbar, q, s, S, U, Pbar, dPdF, rnorm, status, types, R, Kv,
                            restore, args, dev, stream, flush, world, dist)

    if rank != 0:
        dist.destroy_process_group()
        return 0

    # roofline of the dominant kernel (the batched RVE evaluation call:
    # the evaluation kernel and, in the tensor-core form, its condensation
    # kernel), one fraction per execution unit, against peaks measured live
    # on this device by the library's probes
    kinfo = [rv.rve_rom_kernel_info(h, t, args.precision) for t in range(len(roms))]
    n_per_type = np.bincount(types_np, minlength=len(roms))
    w64 = sum(c * work_per_eval(r)[0] for c, r in zip(n_per_type, roms))
    w32 = sum(c * work_per_eval(r)[1] for c, r in zip(n_per_type, roms))
    probe = {u: rv.rverom_peak_probe(u) for u in ('fp32', 'fp64', 'tf32', 'bf16')}
    try:
        hbm_peak, hsrc = json.load(open(os.path.join(ROOT, 'MEASURED_PEAKS.json')))['hbm_gbs'], 'measured copy'
    except (OSError, KeyError, ValueError):
        hbm_peak, hsrc = 6800.0, 'fallback'
    t_s = ms_kern * 1e-3
    traffic = PROFILED_TRAFFIC.get((args.workload, args.precision))
    kname = "; ".join(nm for nm, _ in kinfo) + (" (selected)" if args.candidate >= 0 else " (autotuned)")
    units = {}
    # a5: the reduced-tangent contraction's algorithmic FLOPs (symmetric half
    # plus the Y products) against the tcgen05 TF32 rate
    units["tensor"] = {"achieved": w32 / t_s / 1e12, "peak": probe['tf32'], "unit": "TFLOP/s",
                       "frac": w32 / t_s / 1e12 / probe['tf32'],
                       "peak_source": "measured: tcgen05.mma kind::tf32 probe (rverom_peak_probe)",
                       "work": "a5 contraction, %.0f FLOP per evaluation" % (w32 / n)}
    if args.precision == 'mixed':
        # a2-a4: FP64-accurate kinematics, law and residual as double-float
        # on the FP32 pipe; one double-float multiply-add (2 FLOP) costs 12
        # FP32-pipe instructions, so the pipe's FP64-accurate peak is its
        # FMA rate (2 FLOP per instruction) x 2 / 24
        pk = probe['fp32'] / 12.0
        units["alu"] = {"achieved": w64 / t_s / 1e12, "peak": pk, "unit": "TFLOP/s", "frac": w64 / t_s / 1e12 / pk,
                        "peak_source": "measured FP32 FMA rate %.1f TFLOP/s / 12 (double-float multiply-add: "
                                       "12 FP32 instructions for 2 FLOP)" % probe['fp32'],
                        "work": "a2-a4 FP64-accurate, %.0f FLOP per evaluation" % (w64 / n)}
    else:
        units["alu"] = {"achieved": (w64 + w32) / t_s / 1e12, "peak": probe['fp64'], "unit": "TFLOP/s",
                        "frac": (w64 + w32) / t_s / 1e12 / probe['fp64'],
                        "peak_source": "measured FP64 FMA rate (rverom_peak_probe)",
                        "work": "a2-a5 in float64, %.0f FLOP per evaluation" % ((w64 + w32) / n)}
    if traffic is not None:
        units["hbm"] = {"achieved": traffic / t_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                        "frac": traffic / t_s / 1e9 / hbm_peak, "peak_source": hsrc,
                        "work": "DRAM bytes per launch from an ncu capture of this workload"}
    binding = max(units, key=lambda k: units[k]["frac"])
    head = "tensor" if args.precision == 'mixed' else "alu"
    roofline = dict(units[head])
    roofline.update({"bound": head, "traffic": traffic, "kernel": kname, "kernel_ms": ms_kern,
                     "binding_unit": binding, "units": units, "probe_tflops": probe,
                     "note": "frac is the %s fraction; the unit with the largest fraction (binding_unit) "
                             "limits the kernel" % head})
    cpu = None
    cpu_native = None
    if world == 1 and not args.no_cpu_baseline:
        # the oracle as it stands, one process per host core, on a bounded
        # sample of the workload's points (fresh states at the oracle's own
        # Fbar of the same displacement field), for about 10 s
        from oracle import macro as omacro
        F_or = omacro.MacroMesh(X, conn).gradient(u_host)
        cores = host_cores()
        sel = np.sort(syn.rng(syn.SEED_BASE + 810).choice(n, min(n, 64 * cores), replace=False))
        pool = OraclePool(rom_paths, cores)
        pool.run(types_np[sel][:cores], F_or[sel][:cores])          # workers loaded and warm
        res = pool.run(types_np[sel], F_or[sel], budget=10.0)
        pool.close()
        cnt = sum(c for c, _ in res)
        el = max(e for _, e in res)
        cpu = {"value": cnt / el, "unit": UNIT, "cores": len(res), "kind": "oracle",
               "sample": "%d evaluations in %.1f s on %d processes (one NumPy thread each), each cycling over "
                         "its share of %d sampled points of the %d, fresh micro states; float64 NumPy oracle; "
                         "host %s, %d cores" % (cnt, el, len(res), len(sel), n, cpu_model(), cores)}
        # the plain C++ float64 a1-a7 loop (OpenMP over points) on all host
        # cores and on one, median of 5 runs
        sel_n = syn.rng(syn.SEED_BASE + 811).permutation(n)
        r_all, th_all, np_all = native_cpu_rate(roms, types_np, F_or.reshape(n, -1), sel_n, cores)
        r_one, th_one, np_one = native_cpu_rate(roms, types_np, F_or.reshape(n, -1), sel_n, 1)
        cpu_native = {"kind": "plain C++ float64 a1-a7, OpenMP over points (cpu_baseline/)", "unit": UNIT,
                      "all_cores": {"value": r_all, "threads": th_all, "points_per_run": np_all},
                      "one_core": {"value": r_one, "threads": th_one, "points_per_run": np_one},
                      "statistic": "median of 5 runs", "nproc": cores, "cpu_model": cpu_model()}

    # our kernels per step: gradient, (bucketing: 3 with several types),
    # the evaluation kernels of every type, assembly, norms
    launches = (3 + (3 if len(roms) > 1 else 0) + sum(nl for _, nl in kinfo)) * args.steps
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32" if args.precision == 'mixed' else "f64",
        "data": "synthetic",
        "config": {"workload": args.workload + ': ' + wl['desc'], "macro_points_per_gpu": n,
                   "precision": args.precision, "l2": "flushed between timed steps (256 MB write)",
                   "state": "mid-Newton (converged micro state, q perturbed by 1e-3 |q|)",
                   "autotune_ms": tune,
                   "candidate": args.candidate if args.candidate >= 0 else "autotuned",
                   "failed_points": bad},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "cpu_native": cpu_native,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(u_pin.numel() * 8),
                "d2h_bytes_per_step": int((R_pin.numel() + K_pin.numel() + 3) * 8)},
        "gpu_launches": launches,
        "graph": {"value": graph_value, "ms_per_step": ms_graph,
                  "note": "gradient, evaluation, assembly and norms captured in one CUDA graph"},
        "newton": newton,
        "adjoint": adj,
        "other_workloads": others,
        "clocks": clocks,
        "other_form": {"precision": other, "value": world * n / (ms_other * 1e-3), "ms_per_step": ms_other},
        "speedup_vs_fp64_form": (ms_other / ms_step) if args.precision == 'mixed' else 1.0,
        "accuracy_vs_fp64_form": {"Pbar_rel_err_max": p_err, "dPdF_rel_err_max": c_err,
                                  "Pbar_rel_err_max_per_type": p_err_type,
                                  "points": n, "note": "every point, against the GPU float64 form"},
        "accuracy_vs_oracle": acc,
    }
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


def other_workloads(rv, names, precision, steps, dev, flush):
    """Throughput of the evaluation call on the other workloads (the
    autotuner's kernels, the workload's macro field, the main leg's
    mid-Newton micro states), for the record: evals/s and ms per call, the
    kernels used, and the error of the timed form against the float64 form
    at every point."""
    import torch
    out = {}
    stream = torch.cuda.current_stream()
    for name in names:
        wl = WORKLOADS[name]
        paths = [os.path.join(ROOT, 'tests', 'golden', 'rom_%s.npz' % r) for r in wl['roms']]
        if not all(os.path.exists(p) for p in paths):
            continue
        roms = [rv.load_rom_file(p) for p in paths]
        h = rv.rve_rom_create(wl['d'], roms, roms[0]['V0'])
        rv.rve_rom_autotune(h, precision, n_sample=16384)
        X, conn = build_mesh(wl['mesh'])
        mesh = rv.macro_mesh_create(X, conn)
        n = mesh.n_ip
        types = None
        if len(roms) > 1:
            types = torch.tensor(syn.type_labels(syn.SEED_BASE + 600, n, len(roms)), device=dev)
        u = torch.tensor(macro_displacement(X, wl['load'], syn.SEED_BASE + 500), device=dev)
        Fbar = torch.empty(n, wl['d'] ** 2, dtype=torch.float64, device=dev)
        rv.macro_gradient(mesh, u, Fbar)
        q, s, S, U = h.zero_state(n)
        Pbar, dPdF, rnorm, status = h.outputs(n)
        # the mid-Newton state of the main leg: micro states converged at Fbar
        # by float64 evaluations, then q perturbed by 1e-3 of its size
        for _ in range(4):
            rv.rve_rom_eval_batch(h, Fbar, q, s, S, U, Pbar, dPdF, rnorm, status, type=types, precision='fp64')
        g = torch.Generator(device='cpu').manual_seed(syn.SEED_BASE + 710)
        pert = torch.randn(q.shape, generator=g, dtype=torch.float64).to(dev)
        q += 1e-3 * q.abs().amax(dim=1, keepdim=True) * pert * (q != 0)
        s.zero_()
        S.zero_()
        torch.cuda.synchronize()
        st0 = [x.clone() for x in (q, s, S, U)]
        tot = 0.0
        for _ in range(steps):
            for x, y in zip((q, s, S, U), st0):
                x.copy_(y)
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rv.rve_rom_eval_batch(h, Fbar, q, s, S, U, Pbar, dPdF, rnorm, status, type=types, precision=precision)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        ms = tot / steps
        failed = int((status != 0).sum().item())
        # accuracy at full size: the timed form against the float64 form from
        # the same micro states, every point
        acc = None
        if precision == 'mixed':
            outs = []
            for prec in ('fp64', 'mixed'):
                for x, y in zip((q, s, S, U), st0):
                    x.copy_(y)
                rv.rve_rom_eval_batch(h, Fbar, q, s, S, U, Pbar, dPdF, rnorm, status, type=types, precision=prec)
                outs.append((Pbar.clone(), dPdF.clone(), status.clone()))
            (P64, C64, s64), (Pm, Cm, sm) = outs
            ok = (s64 == 0) & (sm == 0)
            ep = ((Pm - P64).abs().amax(1) / P64.abs().amax(1))[ok]
            ec = ((Cm - C64).abs().amax((1, 2)) / C64.abs().amax((1, 2)))[ok]
            per_type = None
            if types is not None:
                tk = types[ok]
                per_type = {wl['roms'][t]: float(ep[tk == t].max().item()) for t in range(len(roms))}
            acc = {"Pbar_rel_err_max": float(ep.max().item()), "dPdF_rel_err_max": float(ec.max().item()),
                   "Pbar_rel_err_max_per_type": per_type,
                   "Pbar_rel_err_p99": float(torch.quantile(ep.float(), 0.99).item()),
                   "points_over_1e-8": int((ep > 1e-8).sum().item()), "points": int(ok.sum().item()),
                   "against": "float64 GPU form from the same micro states, every point"}
        j2leg = None
        if name == 'c4' and wl['d'] == 2 and len(roms) == 1:
            # the history-dependent law of Example 1 at the ECM points
            # (small-strain J2, yield 0.01 E, hardening 0.016 E in the matrix,
            # elastic inclusions; float64 form), from the same micro states
            # with virgin histories
            mm = rv.rve_rom_mmax(h)
            hin = torch.zeros(n, mm, 7, dtype=torch.float64, device=dev)
            hout = torch.empty_like(hin)
            plastic = np.array([[[0.01, 0.016], [np.inf, 0.0]]])
            tj = 0.0
            for rep in range(4):
                for x, y in zip((q, s, S, U), st0):
                    x.copy_(y)
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rv.rve_rom_eval_batch_j2(h, Fbar, q, s, S, U, hin, hout, plastic, Pbar, dPdF, rnorm, status)
                e1.record(stream)
                e1.synchronize()
                if rep > 0:
                    tj += e0.elapsed_time(e1)
            tj /= 3
            plastic_pts = int((hout[..., 6] > 0).any(dim=1).sum().item())
            j2leg = {"value": n / (tj * 1e-3), "unit": UNIT, "ms_per_call": tj,
                     "failed_points": int((status != 0).sum().item()), "points_yielding": plastic_pts,
                     "form": "float64, one warp per macro point (rve_rom_eval_batch_j2)"}
        out[name] = {"value": n / (ms * 1e-3), "unit": UNIT, "ms_per_call": ms, "points": n,
                     "failed_points": failed, "j2_plasticity": j2leg,
                     "kernels": [rv.rve_rom_kernel_info(h, t, precision)[0] for t in range(len(roms))],
                     "accuracy_vs_fp64_form": acc,
                     "workload": wl['desc'],
                     "state": "mid-Newton (micro states converged by 4 float64 evaluations, q perturbed by 1e-3 |q|)"}
        h.destroy()
        mesh.destroy()
    return out


def newton_leg(rv, h, mesh, wl, u_host, Fbar, q, s, S, U, Pbar, dPdF, rnorm, status, types, R, Kv, restore, args,
               dev, stream, flush, world, dist):
    """Time whole Newton iterations (gradient, evaluation, assembly, norms,
    global solve and update) from the mid-Newton state, prescribed boundary
    DOFs held at the synthetic field's values; also one iteration captured
    in a CUDA graph."""
    import torch
    d = wl['d']
    X, _ = build_mesh(wl['mesh'])
    dofs, _ = meshes.boundary_dofs(wl['mesh'][0], X)
    free_np = np.ones(mesh.n_dof, dtype=np.uint8)
    free_np[dofs] = 0
    free = torch.tensor(free_np, device=dev)
    un = torch.tensor(u_host, device=dev)
    norms = torch.empty(3, dtype=torch.float64, device=dev)
    du = torch.empty(mesh.n_dof, dtype=torch.float64, device=dev)
    K = max(args.steps, 3)
    infos = torch.zeros(args.warmup + K, 3, dtype=torch.float64, device=dev)

    def it(k):
        rv.macro_gradient(mesh, un, Fbar)
        rv.rve_rom_eval_batch(h, Fbar, q, s, S, U, Pbar, dPdF, rnorm, status, type=types, precision=args.precision)
        rv.macro_assemble(mesh, Pbar, dPdF, R, Kv)
        rv.macro_residual_norms(mesh, R, free, rnorm, norms)
        rv.macro_solve(mesh, Kv, R, free, u=un, du=du, info=infos[k], tol=1e-12)

    restore()
    for k in range(args.warmup):
        it(k)
    torch.cuda.synchronize()
    tot, solve_ms = 0.0, 0.0
    for k in range(K):
        flush.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        rv.macro_gradient(mesh, un, Fbar)
        rv.rve_rom_eval_batch(h, Fbar, q, s, S, U, Pbar, dPdF, rnorm, status, type=types, precision=args.precision)
        rv.macro_assemble(mesh, Pbar, dPdF, R, Kv)
        rv.macro_residual_norms(mesh, R, free, rnorm, norms)
        e[1].record(stream)
        rv.macro_solve(mesh, Kv, R, free, u=un, du=du, info=infos[args.warmup + k], tol=1e-12)
        e[2].record(stream)
        e[2].synchronize()
        tot += e[0].elapsed_time(e[2])
        solve_ms += e[1].elapsed_time(e[2])
    inf = infos.cpu().numpy()
    nr = norms.cpu().numpy()
    ms, value = aggregate(tot / K, mesh.n_ip, world, dist, dev)
    out = {"value": value, "unit": UNIT, "ms_per_newton_iteration": ms, "solve_ms": solve_ms / K,
           "iterations_timed": K, "cg_iterations": inf[args.warmup:, 0].astype(int).tolist(),
           "cg_status": inf[args.warmup:, 2].astype(int).tolist(),
           "residual_after": {"R_free_max": float(nr[0]), "R_prescribed_max": float(nr[1]),
                              "micro_r_max": float(nr[2])},
           "bc": "%s: %d prescribed DOFs held at the synthetic field's values" % (wl['mesh'][0], len(dofs)),
           "solve": "macro_solve: block-Jacobi preconditioned CG, relative tolerance 1e-12"}
    # the same Newton iteration captured in one CUDA graph
    try:
        restore()
        un.copy_(torch.tensor(u_host, device=dev))
        it(0)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            with torch.cuda.graph(graph):
                it(0)
        restore()
        un.copy_(torch.tensor(u_host, device=dev))
        torch.cuda.synchronize()
        gms = 0.0
        for _ in range(K):
            flush.zero_()
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            graph.replay()
            g1.record(stream)
            g1.synchronize()
            gms += g0.elapsed_time(g1)
        out["graph_ms_per_newton_iteration"] = gms / K
    except Exception as exc:  # capture of the cooperative launch refused
        out["graph_ms_per_newton_iteration"] = None
        out["graph_note"] = str(exc)[:200]
    restore()
    return out


def run_reference(args, wl, rom_paths, X, conn, u_host):
    """The oracle as it stands on the host cores (one process per core),
    same metric and workload: each step evaluates a bounded sample of the
    workload's macro points (fresh micro states)."""
    from oracle import macro as omacro
    mesh = omacro.MacroMesh(X, conn)
    Fh = mesh.gradient(u_host)
    n = mesh.n_ip
    types = np.zeros(n, dtype=np.int64)
    if len(rom_paths) > 1:
        types = syn.type_labels(syn.SEED_BASE + 600, n, len(rom_paths)).astype(np.int64)
    cores = host_cores()
    per_step = min(n, max(4096, 256 * cores))
    sel = np.arange(0, n, max(1, n // per_step))[:per_step]
    pool = OraclePool(rom_paths, cores)
    for _ in range(args.warmup):
        pool.run(types[sel], Fh[sel])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pool.run(types[sel], Fh[sel])
    el = time.perf_counter() - t0
    pool.close()
    rate = len(sel) * args.steps / el
    sample = ("%d of the %d macro points per step (fresh micro states), float64 NumPy oracle on %d processes "
              "(one NumPy thread each); host %s" % (len(sel), n, cores, cpu_model()))
    out = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": args.workload + ': ' + wl['desc'], "sample_points_per_step": len(sel)},
           "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == '__main__':
    sys.exit(main())
