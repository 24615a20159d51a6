"""GPU parity of the history-dependent evaluation (rve_rom_eval_batch_j2:
small-strain J2 plasticity at the ECM points, Example 1's matrix law)
against the oracle on oracle inputs, and a load-unload macro problem whose
evaluation, assembly and solve run on the GPU against the oracle driver
(irreversible unloading)."""
import numpy as np
import pytest
import torch

import synthetic as syn
from synthetic import meshes
from conftest import rom_path
from oracle import j2, macro, reduced

pytestmark = pytest.mark.gpu
rv = pytest.importorskip('paper_2306_02687_gb300')

PLASTIC = np.array([[[0.01, 0.016], [np.inf, 0.0]]])   # matrix: sy0 = 0.01 E, h = 0.016 E; elastic inclusions


def T(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device='cuda')


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _states(orom, n, seed):
    """Oracle states of a plastic load step: four evaluations at F0 from a
    virgin state; the last records are the converged history; the point is
    then evaluated at a nearby F1."""
    F0 = syn.fbar_batch(seed, 2, n, 0.04, 0.2)
    F1 = F0 + syn.perturbation(seed + 1, F0.shape, 1e-3)
    q = np.zeros((n, orom.n))
    s = np.zeros((n, orom.n))
    S = np.zeros((n, orom.n, 3))
    U = np.zeros((n, 3))
    H = np.zeros((n, orom.m, 7))
    for a in range(n):
        st = reduced.zero_state(orom)
        st['Uprev'] = np.array([1.0, 1.0, 0.0])
        hist = np.zeros((orom.m, 7))
        for _ in range(4):
            o = j2.eval_point(orom, PLASTIC[0], F0[a], hist=hist, **st)
            st = dict(q=o['q'], s=o['s'], S=o['S'], Uprev=o['Uprev'])
        q[a], s[a], S[a], U[a], H[a] = st['q'], st['s'], st['S'], st['Uprev'], o['hist']
        # a mid-Newton state: q perturbed by 1e-3 of its size
        q[a] += syn.perturbation(seed + 7 + a, orom.n, 1e-3 * np.abs(q[a]).max())
    return F1, q, s, S, U, H


@pytest.mark.parametrize('name', ['c1', 'c2'])
def test_j2_evaluation_matches_oracle(name):
    roms = [rv.load_rom_file(rom_path(name))]
    h = rv.rve_rom_create(2, roms, roms[0]['V0'])
    orom = reduced.Rom.load(rom_path(name))
    n = 37 if name == 'c1' else 9
    F, q, s, S, U, H = _states(orom, n, syn.SEED_BASE + 300)
    assert H[..., 6].max() > 0.0                          # some ECM points have yielded
    qd, sd, Sd, Ud = T(q), T(s), T(S), T(U)
    hin, hout = T(H), torch.full((n, orom.m, 7), np.nan, dtype=torch.float64, device='cuda')
    Pbar, dPdF, rnorm, status = h.outputs(n)
    rv.rve_rom_eval_batch_j2(h, T(F.reshape(n, 4)), qd, sd, Sd, Ud, hin, hout, PLASTIC, Pbar, dPdF, rnorm, status)
    torch.cuda.synchronize()
    assert status.max().item() == 0
    g = dict(Pbar=Pbar.cpu().numpy(), dPdF=dPdF.cpu().numpy(), s=sd.cpu().numpy(), S=Sd.cpu().numpy(),
             q=qd.cpu().numpy(), hist=hout.cpu().numpy(), rnorm=rnorm.cpu().numpy())
    for a in range(n):
        o = j2.eval_point(orom, PLASTIC[0], F[a], q[a], s[a], S[a], U[a], H[a])
        assert _rel(g['Pbar'][a], o['Pbar'].ravel()) <= 1e-12
        assert _rel(g['dPdF'][a], o['dPdF']) <= 1e-11
        assert _rel(g['s'][a], o['s']) <= 1e-9 and _rel(g['S'][a], o['S']) <= 1e-9
        assert _rel(g['q'][a], o['q']) <= 1e-12
        assert _rel(g['hist'][a], o['hist']) <= 1e-11
        assert abs(g['rnorm'][a] - o['rnorm']) <= 1e-9 * o['rnorm']
    # a failed point keeps its state and history
    Fb = F.reshape(n, 4).copy()
    Fb[2, 0] = np.nan
    hout2 = torch.zeros_like(hin)
    q2 = T(q)
    rv.rve_rom_eval_batch_j2(h, T(Fb), q2, T(s), T(S), T(U), hin, hout2, PLASTIC, Pbar, dPdF, rnorm, status)
    torch.cuda.synchronize()
    assert status[2].item() == 3 and torch.equal(hout2[2], hin[2]) and torch.equal(q2[2], T(q[2]))


@pytest.mark.parametrize('precision_note', ['fp64'])
def test_load_unload_on_gpu_matches_oracle_driver(precision_note):
    roms = [rv.load_rom_file(rom_path('c1'))]
    h = rv.rve_rom_create(2, roms, roms[0]['V0'])
    orom = reduced.Rom.load(rom_path('c1'))
    X, conn = meshes.rect(2, 2)
    om = macro.MacroMesh(X, conn)
    prob = macro.uniaxial_problem(om, 0.02)
    # unloading in steps of a tenth: the monolithic micro predictor of a
    # larger reversal step overshoots into reverse yielding and cycles
    lf = [0.25, 0.5, 0.75, 1.0, 0.9, 0.8, 0.7, 0.6, 0.5, 0.4, 0.3, 0.2, 0.1, 0.0]
    ref = j2.driver(prob, orom, PLASTIC[0], lf)
    m = rv.macro_mesh_create(X, conn)
    n = m.n_ip
    mm = rv.rve_rom_mmax(h)
    u = torch.zeros(m.n_nodes, 2, dtype=torch.float64, device='cuda')
    q, s, S, U = h.zero_state(n)
    Pbar, dPdF, rnorm, status = h.outputs(n)
    hin = torch.zeros(n, mm, 7, dtype=torch.float64, device='cuda')
    hout = torch.zeros_like(hin)
    Fd = torch.empty(n, 4, dtype=torch.float64, device='cuda')
    R = torch.empty(m.n_dof, dtype=torch.float64, device='cuda')
    Kv = torch.empty(m.nnz, dtype=torch.float64, device='cuda')
    free = np.ones(m.n_dof, dtype=np.uint8)
    free[prob.presc_dofs] = 0
    fr = T(free, torch.uint8)
    norms = torch.empty(3, dtype=torch.float64, device='cuda')
    pidx, pval, react = T(prob.presc_dofs, torch.int64), T(prob.presc_vals), T(prob.react_dofs, torch.int64)
    reactions, iters = [], []
    for lam in lf:
        u.view(-1)[pidx] = lam * pval
        for it in range(31):
            rv.macro_gradient(m, u, Fd)
            rv.rve_rom_eval_batch_j2(h, Fd, q, s, S, U, hin, hout, PLASTIC, Pbar, dPdF, rnorm, status)
            rv.macro_assemble(m, Pbar, dPdF, R, Kv)
            rv.macro_residual_norms(m, R, fr, rnorm, norms)
            nr = norms.cpu().numpy()
            if nr[0] <= 1e-10 * max(1.0, nr[1]) and nr[2] <= 1e-10 * orom.moduli[0, 0] * orom.V0:
                break
            assert it < 30
            rv.macro_solve(m, Kv, R, fr, u=u, tol=1e-13)
        assert status.max().item() == 0
        hin.copy_(hout)                                   # commit the converged history
        reactions.append(R[react].sum().item())
        iters.append(it)
    reactions = np.array(reactions)
    print('reactions', reactions, 'oracle', ref['reactions'])
    assert np.abs(reactions - ref['reactions']).max() <= 1e-9 * np.abs(ref['reactions']).max()
    # histories after 14 converged steps (Newton tolerance 1e-10)
    assert np.abs(hin.cpu().numpy() - ref['hist']).max() <= 1e-8 * np.abs(ref['hist']).max()
    assert abs(reactions[-1]) > 1e-2 * abs(reactions[3])   # irreversible: load remains at zero displacement
    assert max(iters) <= 6
