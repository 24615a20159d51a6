"""The global macro solve on the GPU (macro_solve: block-Jacobi
preconditioned conjugate gradients in one cooperative kernel) against a
direct sparse solve of the same assembled system, its status codes, and a
monolithic Newton loop whose evaluation, assembly, convergence norms and
linear solve all run in the CUDA kernels, against the float64 oracle driver."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import torch

import synthetic as syn
from synthetic import meshes
from conftest import rom_path
from oracle import reduced, macro

pytestmark = pytest.mark.gpu
rv = pytest.importorskip('paper_2306_02687_gb300')


def T(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device='cuda')


def _isotropic_tangent(d, lam, mu):
    """dP/dF of small-strain isotropic elasticity (a positive semi-definite
    stand-in tangent): lam d_iJ d_kL + mu (d_ik d_JL + d_iL d_Jk)."""
    I = np.eye(d)
    C = lam * np.einsum('ij,kl->ijkl', I, I) + mu * (np.einsum('ik,jl->ijkl', I, I) + np.einsum('il,jk->ijkl', I, I))
    return C.reshape(d * d, d * d)


def _system(kind):
    if kind == 'rect':
        X, conn = meshes.rect(12, 7, 1.5, 1.0)
    elif kind == 'plate':
        X, conn = meshes.plate_with_hole(16, 16)
    else:
        X, conn = meshes.box(6, 5, 3, 1.0, 1.0, 0.5)
    d = X.shape[1]
    m = rv.macro_mesh_create(X, conn)
    g = d * d
    # per-point tangent: isotropic elasticity with seeded per-point moduli
    r = syn.rng(syn.SEED_BASE + 60)
    C = np.array([_isotropic_tangent(d, 0.5 + r.random(), 0.3 + r.random()) for _ in range(m.n_ip)])
    P = syn.perturbation(syn.SEED_BASE + 61, (m.n_ip, g), 0.1)
    R = torch.empty(m.n_dof, dtype=torch.float64, device='cuda')
    Kv = torch.empty(m.nnz, dtype=torch.float64, device='cuda')
    rv.macro_assemble(m, T(P), T(C), R, Kv)
    # prescribed: every DOF of the nodes on the plane/line X_0 = min, plus
    # the second DOF of the nodes at X_1 = min (rigid motions removed)
    free = np.ones(m.n_dof, dtype=np.uint8)
    x0 = np.isclose(X[:, 0], X[:, 0].min())
    for i in range(d):
        free[np.nonzero(x0)[0] * d + i] = 0
    free[np.nonzero(np.isclose(X[:, 1], X[:, 1].min()))[0] * d + 1] = 0
    return m, X, R, Kv, free


@pytest.mark.parametrize('kind', ['rect', 'plate', 'box'])
def test_macro_solve_matches_direct_solve(kind):
    m, X, R, Kv, free = _system(kind)
    u0 = syn.perturbation(syn.SEED_BASE + 62, X.shape, 0.01)
    u = T(u0)
    du, info = rv.macro_solve(m, Kv, R, T(free, torch.uint8), u=u, tol=1e-14)
    torch.cuda.synchronize()
    it, res, status = info.cpu().numpy()
    assert status == 0 and res <= 1e-14 and 0 < it < 20000
    rp, col = m.csr()
    K = sp.csr_matrix((Kv.cpu().numpy(), col, rp), shape=(m.n_dof, m.n_dof))
    fi = np.nonzero(free)[0]
    ref = spla.spsolve(K[fi][:, fi].tocsc(), -R.cpu().numpy()[fi])
    got = du.cpu().numpy()
    print(kind, 'n_dof', m.n_dof, 'iterations', int(it))
    assert np.abs(got[fi] - ref).max() <= 1e-9 * np.abs(ref).max()
    assert np.all(got[free == 0] == 0.0)
    assert np.array_equal(u.cpu().numpy().ravel(), u0.ravel() + got)


def test_macro_solve_status_codes():
    m, X, R, Kv, free = _system('rect')
    fr = T(free, torch.uint8)
    du, info = rv.macro_solve(m, Kv, R, fr, tol=1e-14, max_iter=1)
    torch.cuda.synchronize()
    it, res, status = info.cpu().numpy()
    assert status == 1 and it == 1 and res > 1e-14
    du, info = rv.macro_solve(m, Kv, torch.zeros_like(R), fr, tol=1e-14)
    torch.cuda.synchronize()
    assert list(info.cpu().numpy()) == [0.0, 0.0, 0.0] and torch.all(du == 0)
    # a negative definite system: breakdown on the first search direction
    du, info = rv.macro_solve(m, -Kv, R, fr, tol=1e-14)
    torch.cuda.synchronize()
    assert info.cpu().numpy()[2] == 2
    # repeated calls on one mesh give the same result
    d1, i1 = rv.macro_solve(m, Kv, R, fr, tol=1e-12)
    d1 = d1.clone()
    d2, i2 = rv.macro_solve(m, Kv, R, fr, tol=1e-12)
    torch.cuda.synchronize()
    assert torch.equal(d1, d2)


@pytest.mark.parametrize('precision', ['fp64', 'mixed'])
def test_monolithic_newton_fully_on_gpu(precision):
    """Uniaxial tension of a 4x4 Q4 square (64 macro points) with the
    16x16 / 12-mode / 60-point ROM to 10% in 10 load steps, tolerance 1e-10:
    every evaluation, assembly, norm and linear solve on the GPU (the host
    only reads the three convergence scalars); the reactions and the
    displacements match the float64 oracle driver."""
    roms = [rv.load_rom_file(rom_path('c1'))]
    h = rv.rve_rom_create(2, roms, roms[0]['V0'])
    orom = reduced.Rom.load(rom_path('c1'))
    X, conn = meshes.rect(4, 4)
    m = rv.macro_mesh_create(X, conn)
    om = macro.MacroMesh(X, conn)
    prob = macro.uniaxial_problem(om, 0.1)
    n_steps = 10
    ref = macro.driver(prob, [orom], np.zeros(om.n_ip, dtype=np.int64), n_steps)
    n = m.n_ip
    u = torch.zeros(m.n_nodes, 2, dtype=torch.float64, device='cuda')
    q, s, S, U = h.zero_state(n)
    Pbar, dPdF, rnorm, status = h.outputs(n)
    Fd = torch.empty(n, 4, dtype=torch.float64, device='cuda')
    R = torch.empty(m.n_dof, dtype=torch.float64, device='cuda')
    Kv = torch.empty(m.nnz, dtype=torch.float64, device='cuda')
    free = np.ones(m.n_dof, dtype=np.uint8)
    free[prob.presc_dofs] = 0
    fr = T(free, torch.uint8)
    norms = torch.empty(3, dtype=torch.float64, device='cuda')
    pidx = T(prob.presc_dofs, torch.int64)
    pval = T(prob.presc_vals)
    react = T(prob.react_dofs, torch.int64)
    reactions, iters, cg = [], [], []
    mu_m = orom.moduli[0, 0]
    for step in range(1, n_steps + 1):
        u.view(-1)[pidx] = step / n_steps * pval          # load step: prescribed values
        for it in range(31):
            rv.macro_gradient(m, u, Fd)
            rv.rve_rom_eval_batch(h, Fd, q, s, S, U, Pbar, dPdF, rnorm, status, precision=precision)
            rv.macro_assemble(m, Pbar, dPdF, R, Kv)
            rv.macro_residual_norms(m, R, fr, rnorm, norms)
            nr = norms.cpu().numpy()                       # the host reads three scalars
            if nr[0] <= 1e-10 * max(1.0, nr[1]) and nr[2] <= 1e-10 * mu_m * orom.V0:
                break
            assert it < 30
            _, info = rv.macro_solve(m, Kv, R, fr, u=u, tol=1e-13)
            cg.append(info.cpu().numpy())
        assert status.max().item() == 0
        reactions.append(R[react].sum().item())
        iters.append(it)
    cg = np.array(cg)
    print(precision, 'Newton iterations', iters, 'CG iterations', cg[:, 0].astype(int).tolist())
    assert np.all(cg[:, 2] == 0)
    assert max(iters) <= 6
    assert np.abs(np.array(reactions) - ref['reactions']).max() <= 1e-9 * np.abs(ref['reactions']).max()
    assert np.abs(u.cpu().numpy() - ref['u']).max() <= 1e-9
