"""Parity at the full sizes of the other workloads, in the launch
configuration the benchmark times (the autotuner's pick per RVE type):
  c4  16 384 points of the 12-mode ROM,
  c3  65 536 points of the 3D 40-mode ROM,
  c5  131 044 points of three ROM types (16, 32, 64 modes) mixed at random.
Sampled points carry oracle mid-Newton states and are compared with the
float64 oracle one by one at the mixed-form gate; every point whose micro
iteration converged is compared with the float64 GPU form from the same
micro states (stress 1e-8, tangent 1e-5 relative, per point)."""
import numpy as np
import pytest
import torch

import synthetic as syn
from conftest import rom_path
from test_gpu_eval import _handle, compare, mid_newton_inputs, oracle_batch, TOL_MIXED

pytestmark = pytest.mark.gpu
rv = pytest.importorskip('paper_2306_02687_gb300')

CASES = {
    'c4': (['c1'], 16384, 0.1),
    'c3': (['c3'], 65536, 0.2),
    'c5': (['c5a', 'c5b', 'c5c'], 131044, 0.14),
}


@pytest.mark.parametrize('case', ['c4', 'c3', 'c5'])
def test_full_size_sampled(case):
    import os
    names, n, eps = CASES[case]
    if not all(os.path.exists(rom_path(nm)) for nm in names):
        pytest.skip('ROM files not generated')
    h, oroms = _handle(names)
    d = oroms[0].d
    ns = oroms[0].ns
    dev = 'cuda'
    types = syn.type_labels(syn.SEED_BASE + 90, n, len(names)) if len(names) > 1 else None
    ty = None if types is None else torch.tensor(types, dtype=torch.int32, device=dev)
    F = syn.fbar_batch(syn.SEED_BASE + 91, d, n, eps, 0.3).reshape(n, d * d)
    # mid-Newton states everywhere: micro states converged by float64
    # evaluations, then q perturbed by 1e-3 of its size
    Fd = torch.tensor(F, device=dev)
    q, s, S, U = h.zero_state(n)
    Pbar, dPdF, rnorm, status = h.outputs(n)
    for _ in range(8):
        rv.rve_rom_eval_batch(h, Fd, q, s, S, U, Pbar, dPdF, rnorm, status, type=ty, precision='fp64')
    # points whose micro iteration converged: the random stretches include
    # volumetric compression to det F = 0.83, beyond the training range of
    # the 64-mode ROM, where its micro Newton iteration folds ECM points and
    # wanders (c5: about 220 of 131 044 points; the oracle's own micro solve
    # fails there too).  Those stay in the batch but are not mid-Newton
    # states of a converging iteration, the states the stress gate is for.
    conv = ((status == 0) & (rnorm <= 1e-8)).cpu().numpy()
    print(case, 'converged micro states: %d of %d' % (conv.sum(), n))
    assert conv.mean() >= 0.98
    g = torch.Generator(device='cpu').manual_seed(syn.SEED_BASE + 92)
    pert = torch.randn(q.shape, generator=g, dtype=torch.float64).to(dev)
    q += 1e-3 * q.abs().amax(dim=1, keepdim=True) * pert * (q != 0)
    s.zero_()
    S.zero_()
    # sampled points: states the oracle converged (their inputs come from
    # the oracle only)
    per_type = 12 if len(names) > 1 else 24
    idx_all, o_all = [], []
    for t in range(len(names)):
        cand = np.arange(n) if types is None else np.nonzero(types == t)[0]
        idx = np.sort(syn.rng(syn.SEED_BASE + 93 + t).choice(cand, per_type, replace=False))
        Fm, qm, sm, Sm, Um = mid_newton_inputs(oroms[t], per_type, syn.SEED_BASE + 94 + 10 * t, eps=eps)
        k = oroms[t].n
        it = torch.tensor(idx, device=dev)
        Fd[it] = torch.tensor(Fm.reshape(per_type, -1), device=dev)
        qn = np.zeros((per_type, h.nmax))
        sn = np.zeros((per_type, h.nmax))
        Sn = np.zeros((per_type, h.nmax, ns))
        qn[:, :k], sn[:, :k], Sn[:, :k] = qm, sm, Sm
        q[it], s[it], S[it], U[it] = (torch.tensor(x, device=dev) for x in (qn, sn, Sn, Um))
        conv[idx] = True
        idx_all.append(idx)
        o_all.append((Fm, qn, sn, Sn, Um))
    state0 = [x.clone() for x in (q, s, S, U)]

    def run(precision):
        for x, y in zip((q, s, S, U), state0):
            x.copy_(y)
        rv.rve_rom_eval_batch(h, Fd, q, s, S, U, Pbar, dPdF, rnorm, status, type=ty, precision=precision)
        torch.cuda.synchronize()
        return dict(Pbar=Pbar.cpu().numpy(), dPdF=dPdF.cpu().numpy(), rnorm=rnorm.cpu().numpy(),
                    status=status.cpu().numpy(), q=q.cpu().numpy(), s=s.cpu().numpy(), S=S.cpu().numpy(),
                    Uprev=U.cpu().numpy())

    ref = run('fp64')
    ms = rv.rve_rom_autotune(h, 'mixed', n_sample=16384)
    assert np.all(ms[:, 0] > 0)
    kernels = [rv.rve_rom_kernel_info(h, t, 'mixed')[0] for t in range(len(names))]
    print(case, 'autotuned:', kernels)
    got = run('mixed')
    for nm, r in (('float64', ref), ('mixed', got)):
        vals, cnt = np.unique(r['status'], return_counts=True)
        print(case, nm, 'status counts', dict(zip(vals.tolist(), cnt.tolist())))
    # at some of the points whose micro iteration did not converge the
    # reduced stiffness is not positive definite (c5: 111 points, status 2):
    # both forms must report the same points
    assert np.array_equal(ref['status'], got['status'])
    ok = (ref['status'] == 0) & conv
    assert ok.mean() >= 0.98
    # every other point against the float64 form
    ep = (np.abs(got['Pbar'] - ref['Pbar']).max(axis=1) / np.abs(ref['Pbar']).max(axis=1))[ok]
    ec = (np.abs(got['dPdF'] - ref['dPdF']).max(axis=(1, 2)) / np.abs(ref['dPdF']).max(axis=(1, 2)))[ok]
    print(case, 'vs float64 form: Pbar max %.2e p99 %.2e, dPdF max %.2e' % (ep.max(), np.quantile(ep, 0.99),
                                                                         ec.max()))
    if types is not None:
        print(case, 'Pbar max per type', [float(ep[types[ok] == t].max()) for t in range(len(names))])
        print(case, 'excluded per type', [int(((types == t) & ~ok).sum()) for t in range(len(names))])
    assert ep.max() <= 1e-8 and ec.max() <= 1e-5
    # sampled points against the oracle
    for t in range(len(names)):
        Fm, qn, sn, Sn, Um = o_all[t]
        tt = None if types is None else np.full(per_type, t)
        outs = oracle_batch(oroms, Fm, qn, sn, Sn, Um, tt)
        idx = idx_all[t]
        compare({k: v[idx] for k, v in got.items()}, outs, h.nmax, TOL_MIXED)
