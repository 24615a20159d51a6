"""GPU parity of the offline stage (Sec. 3.2.1 snapshots and POD, Sec. 3.3
empirical cubature) against the oracle's offline functions, on oracle
inputs (RVE geometry, phases, seeded training paths)."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import law, rom, rve

pytestmark = pytest.mark.gpu
rv = pytest.importorskip('paper_2306_02687_gb300')
from paper_2306_02687_gb300 import offline  # noqa: E402

MOD = np.array([law.mu_kappa_from_E_nu(1.0, 0.3), law.mu_kappa_from_E_nu(10.0, 0.3)])


def _model(n, vf=0.2):
    return rve.PeriodicRVE(2, n, rve.phases_single_inclusion(2, n, vf), MOD)


def test_snapshots_and_linear_responses_match_oracle():
    n = 12
    m = _model(n)
    paths = syn.training_paths(syn.SEED_BASE + 310, 2, 5, 4, 0.12)
    X_or = rom.snapshots(m, paths)                         # [n_dof, n_snap]
    X, info = offline.rve_snapshots(n, m.phase, MOD, torch.tensor(paths, device='cuda'))
    torch.cuda.synchronize()
    inf = info.cpu().numpy()
    assert np.all(inf[:, 3] == 0), inf
    Xg = X.cpu().numpy().T
    err = np.abs(Xg - X_or).max() / np.abs(X_or).max()
    print('snapshots: max rel err %.2e, Newton %s, CG %s' % (err, inf[:, 0], inf[:, 1]))
    assert err <= 1e-8
    W_or = m.linear_responses()                            # [n_dof, 3]
    W, info = offline.rve_snapshots(n, m.phase, MOD, linear=True, cg_tol=1e-14)
    torch.cuda.synchronize()
    assert np.all(info.cpu().numpy()[:, 3] == 0)
    assert np.abs(W.cpu().numpy().T - W_or).max() <= 1e-10 * np.abs(W_or).max()


def test_offline_pipeline_matches_oracle():
    # the whole offline stage on the GPU (snapshots, linearized responses,
    # POD, fully integrated ROM runs, ECM training matrix, empirical
    # cubature) against the oracle's on the same RVE and training paths
    n, n_modes, m_target = 16, 8, 30
    model = _model(n)
    paths = syn.training_paths(syn.SEED_BASE + 320, 2, 8, 4, 0.1)
    X_or = rom.snapshots(model, paths)
    Phi_or = rom.pod_basis(model, X_or, n_modes)
    fk = rom.ecm_training(model, Phi_or, paths)
    xf_or = rom.training_matrix(fk, model.ip_weight, model.V0, n_modes)
    z_or, w_or = rom.ecm(xf_or, model.V0, m_target)
    rom_g, st = offline.build_hyper_rom(n, model.phase, MOD, paths, n_modes, m_target,
                                        rng=syn.rng(syn.SEED_BASE + 321))
    print('times', st['times'], 'ecm info', st['info_ecm'], 'pod info', st['info_pod'])
    assert np.all(st['info_snap'][:, 3] == 0) and np.all(st['info_lin'][:, 3] == 0)
    Phi = st['Phi'].cpu().numpy().T                         # [n_dof, n_modes]
    # the elastic modes span the oracle's; the whole basis too (the
    # spectrum has a gap at the truncation)
    P_el = Phi[:, :3] @ Phi[:, :3].T
    assert np.abs(P_el - Phi_or[:, :3] @ Phi_or[:, :3].T).max() <= 1e-10
    eig = st['eig'].cpu().numpy()
    k = n_modes - 3
    assert eig[k] < 0.5 * eig[k - 1]
    assert np.abs(Phi @ Phi.T - Phi_or @ Phi_or.T).max() <= 1e-7
    # the training matrix up to the rotation of the modes: x_f^T x_f
    xf = st['xf'].cpu().numpy()
    Gg, Go = xf.T @ xf, xf_or.T @ xf_or
    assert np.abs(Gg - Go).max() <= 1e-6 * np.abs(Go).max()
    # empirical cubature, randomized range finder (the pipeline's default):
    # valid weights on the volume; the selection need not be the oracle's
    # (Box 1 on an approximate singular subspace), its accuracy is checked below
    z, w = st['z'], rom_g['w']
    assert np.all(w > 0) and abs(w.sum() - 1.0) <= 1e-8 and len(z) <= m_target
    common = len(set(z.tolist()) & set(z_or.tolist()))
    print('ECM points (randomized): gpu %d, oracle %d, common %d' % (len(z), len(z_or), common))
    # Box 1 on the oracle's training matrix: the GPU's x_f agrees with the
    # oracle's only to the accuracy of the POD basis (the Gram matrices to
    # 1e-6), which can turn the 29-dimensional singular subspace by more than
    # the greedy's margins; on the same x_f both the randomized range finder
    # (k = 39, two power iterations) and the whole row space (k = n_rows)
    # give the oracle's singular subspace and points; the weights to the
    # accuracy of that subspace (randomized: of order (sigma_40 /
    # sigma_29)^5 ~ 1e-3 relative, amplified by the conditioning of the
    # 30 x 30 least-squares system; whole row space: rounding of the Gram
    # eigenproblem, ~1e-12, amplified the same way)
    n_rows = xf_or.shape[0]
    xo = torch.tensor(np.ascontiguousarray(xf_or), device='cuda').contiguous()
    for k, its, wtol in ((m_target - 1 + 10, 2, 1e-4), (n_rows, 0, 1e-6)):
        Om = torch.tensor(syn.rng(syn.SEED_BASE + 323).standard_normal((n_rows, k)), device='cuda')
        ze, we, ie = offline.ecm_select(xo, 1.0, m_target, Om, power_its=its)
        print('ECM on the oracle x_f, k %d: info %s, common %d' % (k, ie, len(set(ze.tolist()) & set(z_or.tolist()))))
        oe, oo = np.argsort(ze), np.argsort(z_or)
        assert np.array_equal(ze[oe], z_or[oo])
        assert np.abs(we[oe] - w_or[oo]).max() <= wtol * w_or.max()
    # the GPU-built hyper-ROM against the oracle-built one and the fully
    # integrated ROM at a test stretch
    from oracle import reduced
    rg = reduced.Rom(rom_g['B'], rom_g['w'], rom_g['phase'], rom_g['moduli'], 1.0)
    ro = rom.hyper_rom(model, Phi_or, z_or, w_or)
    rf = rom.full_integration_rom(model, Phi_or)
    Fb = syn.fbar_batch(syn.SEED_BASE + 322, 2, 1, 0.08, 0.0)[0]
    Pg = reduced.converge_point(rg, Fb)[0]['Pbar']
    Po = reduced.converge_point(ro, Fb)[0]['Pbar']
    Pf = reduced.converge_point(rf, Fb)[0]['Pbar']
    eo, eg = np.abs(Po - Pf).max(), np.abs(Pg - Pf).max()
    print('hyper-ROM error vs full integration: oracle %.2e, gpu %.2e' % (eo, eg))
    assert eg <= max(3 * eo, 1e-6 * np.abs(Pf).max())


def test_offline_stage_at_the_24_mode_scale():
    # the offline stage on the GPU for the RVE of the 24-mode workload (48 x 48
    # Q4, four seeded inclusions, 20 training paths x 10 steps up to 0.15, 24
    # modes, 200 ECM points: the recipe of the stored ROM, which the oracle
    # built); the GPU-built hyper-ROM must approximate the full-order RVE as
    # well as the oracle-built one at seeded test stretches
    import importlib.util
    import os
    from oracle import reduced
    from conftest import rom_path
    here = os.path.dirname(os.path.abspath(__file__))
    spec = importlib.util.spec_from_file_location('make_roms', os.path.join(here, 'golden', 'make_roms.py'))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    c = mk.CONFIGS['c2']
    model = mk.build_rve(c)
    paths = syn.training_paths(syn.SEED_BASE + c['seed'], 2, c['paths'], c['steps'], c['eps'])
    rom_g, st = offline.build_hyper_rom(c['n'], model.phase, MOD, paths, c['modes'], c['ecm'],
                                        rng=syn.rng(syn.SEED_BASE + 330))
    print('48 x 48 RVE offline stage on the GPU:', {k: round(v, 3) for k, v in st['times'].items()},
          'ECM points', len(rom_g['w']), 'ecm info', st['info_ecm'])
    assert np.all(st['info_snap'][:, 3] == 0) and np.all(st['info_lin'][:, 3] == 0)
    w = rom_g['w']
    assert np.all(w > 0) and abs(w.sum() - 1.0) <= 1e-8 and 100 <= len(w) <= c['ecm']
    rg = reduced.Rom(rom_g['B'], w, rom_g['phase'], rom_g['moduli'], 1.0)
    ro = reduced.Rom.load(rom_path('c2'))
    Fs = syn.fbar_batch(syn.SEED_BASE + 331, 2, 3, 0.1, 0.3)
    for Fb in Fs:
        Pf = model.solve(Fb)[1]
        Pg = reduced.converge_point(rg, Fb)[0]['Pbar']
        Po = reduced.converge_point(ro, Fb)[0]['Pbar']
        eg, eo = np.abs(Pg - Pf).max() / np.abs(Pf).max(), np.abs(Po - Pf).max() / np.abs(Pf).max()
        print('hyper-ROM error against the full-order RVE: GPU-built %.2e, oracle-built %.2e' % (eg, eo))
        assert eg <= max(3 * eo, 5e-3)
