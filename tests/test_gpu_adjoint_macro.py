"""GPU parity of rve_rom_adjoint, macro_gradient, macro_assemble and
macro_residual_norms against the CPU oracle, and a monolithic Newton loop
whose every evaluation and assembly runs in the CUDA kernels (the linear
solve of the assembled macro system is done by the test on the host)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import torch

import synthetic as syn
from synthetic import meshes
from conftest import rom_path
from oracle import reduced, adjoint, macro

pytestmark = pytest.mark.gpu
rv = pytest.importorskip('paper_2306_02687_gb300')


def _handle(names):
    roms = [rv.load_rom_file(rom_path(nm)) for nm in names]
    d = int(round(np.sqrt(roms[0]['B'].shape[1])))
    return rv.rve_rom_create(d, roms, roms[0]['V0']), [reduced.Rom.load(rom_path(nm)) for nm in names]


def T(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device='cuda')


def test_adjoint_matches_oracle():
    h, oroms = _handle(['c1'])
    n = 21
    F = syn.fbar_batch(syn.SEED_BASE + 40, 2, n, 0.1, 0.4)
    q = np.zeros((n, h.nmax))
    for a in range(n):
        o, _ = reduced.converge_point(oroms[0], F[a])
        q[a] = o['q']
    gP = syn.perturbation(syn.SEED_BASE + 41, (n, 4), 1.0)
    gF = torch.empty(n, 4, dtype=torch.float64, device='cuda')
    gth = torch.zeros(1, 2, 2, dtype=torch.float64, device='cuda')
    status = torch.empty(n, dtype=torch.int32, device='cuda')
    rv.rve_rom_adjoint(h, T(F.reshape(n, 4)), T(q), T(gP), gF, gth, status)
    torch.cuda.synchronize()
    assert status.max().item() == 0
    gth_o = np.zeros((2, 2))
    gFo = np.zeros((n, 4))
    for a in range(n):
        gf, gt = adjoint.point_adjoint(oroms[0], F[a], q[a], gP[a])
        gFo[a] = gf
        gth_o += gt
    assert np.abs(gF.cpu().numpy() - gFo).max() <= 1e-11 * np.abs(gFo).max()
    assert np.abs(gth.cpu().numpy()[0] - gth_o).max() <= 1e-10 * np.abs(gth_o).max()
    # accumulation: a second call adds the same amount
    rv.rve_rom_adjoint(h, T(F.reshape(n, 4)), T(q), T(gP), gF, gth, status)
    torch.cuda.synchronize()
    assert np.abs(gth.cpu().numpy()[0] - 2 * gth_o).max() <= 2e-10 * np.abs(gth_o).max()


def test_adjoint_mixed_types_and_fd():
    import os
    names = ['c5a', 'c5b', 'c5c']
    if not all(os.path.exists(rom_path(nm)) for nm in names):
        pytest.skip('mixed-type ROM files not generated')
    h, oroms = _handle(names)
    n = 18
    types = syn.type_labels(syn.SEED_BASE + 42, n, 3)
    F = syn.fbar_batch(syn.SEED_BASE + 43, 2, n, 0.12, 0.3)
    q = np.zeros((n, h.nmax))
    for a in range(n):
        o, _ = reduced.converge_point(oroms[types[a]], F[a])
        q[a, :oroms[types[a]].n] = o['q']
    gP = syn.perturbation(syn.SEED_BASE + 44, (n, 4), 1.0)
    gF = torch.empty(n, 4, dtype=torch.float64, device='cuda')
    gth = torch.zeros(3, 2, 2, dtype=torch.float64, device='cuda')
    status = torch.empty(n, dtype=torch.int32, device='cuda')
    rv.rve_rom_adjoint(h, T(F.reshape(n, 4)), T(q), T(gP), gF, gth, status, type=T(types, torch.int32))
    torch.cuda.synchronize()
    ref = np.zeros((3, 2, 2))
    for a in range(n):
        r = oroms[types[a]]
        _, gt = adjoint.point_adjoint(r, F[a], q[a, :r.n], gP[a])
        ref[types[a]] += gt
    got = gth.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


def _macro_pair(X, conn):
    return rv.macro_mesh_create(X, conn), macro.MacroMesh(X, conn)


@pytest.mark.parametrize('kind', ['rect', 'plate', 'box'])
def test_macro_gradient_assembly_norms(kind):
    if kind == 'rect':
        X, conn = meshes.rect(5, 3, 1.5, 1.0)
    elif kind == 'plate':
        X, conn = meshes.plate_with_hole(4, 4)
    else:
        X, conn = meshes.box(3, 2, 2, 1.0, 1.0, 0.5)
    m, om = _macro_pair(X, conn)
    d = X.shape[1]
    g = d * d
    u = syn.perturbation(syn.SEED_BASE + 45, X.shape, 0.02)
    Fd = torch.empty(m.n_ip, g, dtype=torch.float64, device='cuda')
    rv.macro_gradient(m, T(u), Fd)
    Fo = om.gradient(u)
    assert np.abs(Fd.cpu().numpy() - Fo.reshape(-1, g)).max() < 1e-14
    P = syn.perturbation(syn.SEED_BASE + 46, (m.n_ip, g), 1.0)
    C = syn.perturbation(syn.SEED_BASE + 47, (m.n_ip, g, g), 1.0)
    R = torch.empty(m.n_dof, dtype=torch.float64, device='cuda')
    Kv = torch.empty(m.nnz, dtype=torch.float64, device='cuda')
    rv.macro_assemble(m, T(P), T(C), R, Kv)
    Ro, Ko = om.assemble(P.reshape(-1, d, d), C)
    assert np.abs(R.cpu().numpy() - Ro).max() <= 1e-13 * np.abs(Ro).max()
    rp, col = m.csr()
    Kg = sp.csr_matrix((Kv.cpu().numpy(), col, rp), shape=(m.n_dof, m.n_dof)).toarray()
    assert np.abs(Kg - Ko.toarray()).max() <= 1e-13 * np.abs(Ko).max()
    # residual-only assembly
    R2 = torch.empty_like(R)
    rv.macro_assemble(m, T(P), None, R2, None)
    assert torch.equal(R, R2) or (R - R2).abs().max().item() < 1e-13
    free = np.ones(m.n_dof, dtype=np.uint8)
    free[:d] = 0
    rn = syn.perturbation(syn.SEED_BASE + 48, (7,), 1.0) ** 2
    out = torch.empty(3, dtype=torch.float64, device='cuda')
    rv.macro_residual_norms(m, T(Ro), T(free, torch.uint8), T(rn), out)
    exp = [np.abs(Ro[free == 1]).max(), np.abs(Ro[free == 0]).max(), rn.max()]
    assert np.allclose(out.cpu().numpy(), exp, rtol=0, atol=0)


@pytest.mark.parametrize('precision', ['fp64', 'mixed'])
def test_monolithic_newton_on_gpu_matches_oracle(precision):
    """Uniaxial tension of a 3x3 Q4 square with the 16x16/12-mode ROM: every
    RVE evaluation, F, R and K come from the CUDA kernels; the converged
    reactions match the float64 oracle driver."""
    h, oroms = _handle(['c1'])
    X, conn = meshes.rect(3, 3)
    m, om = _macro_pair(X, conn)
    prob = macro.uniaxial_problem(om, 0.1)
    n_steps = 4
    ref = macro.driver(prob, oroms, np.zeros(om.n_ip, dtype=np.int64), n_steps)
    n = m.n_ip
    u = np.zeros((m.n_nodes, 2))
    q, s, S, U = h.zero_state(n)
    Pbar, dPdF, rnorm, status = h.outputs(n)
    Fd = torch.empty(n, 4, dtype=torch.float64, device='cuda')
    R = torch.empty(m.n_dof, dtype=torch.float64, device='cuda')
    Kv = torch.empty(m.nnz, dtype=torch.float64, device='cuda')
    rp, col = m.csr()
    reactions, iters = [], []
    for step in range(1, n_steps + 1):
        uf = u.reshape(-1)
        uf[prob.presc_dofs] = step / n_steps * prob.presc_vals
        for it in range(30):
            rv.macro_gradient(m, T(u), Fd)
            rv.rve_rom_eval_batch(h, Fd, q, s, S, U, Pbar, dPdF, rnorm, status, precision=precision)
            rv.macro_assemble(m, Pbar, dPdF, R, Kv)
            torch.cuda.synchronize()
            assert status.max().item() == 0
            Rh = R.cpu().numpy()
            Rf = Rh[prob.free]
            if (np.abs(Rf).max() <= 1e-10 * max(1.0, np.abs(Rh[prob.presc_dofs]).max())
                    and rnorm.max().item() <= 1e-10 * oroms[0].moduli[0, 0]):
                break
            K = sp.csr_matrix((Kv.cpu().numpy(), col, rp), shape=(m.n_dof, m.n_dof)).tocsc()
            du = spla.spsolve(K[prob.free][:, prob.free], -Rf)
            uf = u.reshape(-1)
            uf[prob.free] += du
        reactions.append(Rh[prob.react_dofs].sum())
        iters.append(it)
    assert max(iters) <= 5
    assert np.abs(np.array(reactions) - ref['reactions']).max() <= 1e-9 * np.abs(ref['reactions']).max()
    assert np.abs(u - ref['u']).max() <= 1e-9


def test_autograd_function_against_oracle():
    h, oroms = _handle(['c1'])
    n = 12
    F = syn.fbar_batch(syn.SEED_BASE + 49, 2, n, 0.1, 0.3)
    W = syn.perturbation(syn.SEED_BASE + 50, (n, 4), 1.0)
    Fd = T(F.reshape(n, 4)).requires_grad_(True)
    mod = torch.tensor(oroms[0].moduli[None], dtype=torch.float64, device='cuda', requires_grad=True)
    P = rv.rve_stress(Fd, mod, h)
    L = (P * T(W)).sum()
    L.backward()
    gth_o = np.zeros((2, 2))
    for a in range(n):
        o, _ = reduced.converge_point(oroms[0], F[a])
        assert np.abs(P.detach().cpu().numpy()[a] - o['Pbar'].ravel()).max() <= 1e-11
        gf, gt = adjoint.point_adjoint(oroms[0], F[a], o['q'], W[a])
        assert np.abs(Fd.grad.cpu().numpy()[a] - gf).max() <= 1e-10 * np.abs(gf).max()
        gth_o += gt
    assert np.abs(mod.grad.cpu().numpy()[0] - gth_o).max() <= 1e-9 * np.abs(gth_o).max()


def test_reaction_loss_gradient_chain_on_gpu():
    """d(sum_steps (reaction - target)^2)/d(moduli) with the evaluation,
    assembly and per-point adjoint on the GPU and the macro adjoint solve on
    the host; compared with the oracle's gradient and with central finite
    differences of the oracle loss."""
    h, oroms = _handle(['c1'])
    orom = oroms[0]
    X, conn = meshes.rect(2, 2)
    m, om = _macro_pair(X, conn)
    prob = macro.uniaxial_problem(om, 0.1)
    ns = 3
    g = syn.rng(syn.SEED_BASE + 4)
    scale = 0.8 + 0.4 * g.random((2, 2))
    target = np.array([st[0] for st in adjoint.driver_steps(prob, orom.with_moduli(orom.moduli * scale), ns, 1e-12)])
    L_o, grad_o = adjoint.reaction_loss_and_grad(prob, orom, ns, target)
    # GPU: converged states per step from the oracle driver's displacements,
    # micro equilibrium and cotangents from the GPU kernels
    steps = adjoint.driver_steps(prob, orom, ns, 1e-12)
    grad = torch.zeros(1, 2, 2, dtype=torch.float64, device='cuda')
    n = m.n_ip
    rp, col = m.csr()
    for k, (reac, u_n, K_n, qs) in enumerate(steps):
        Fd = torch.empty(n, 4, dtype=torch.float64, device='cuda')
        rv.macro_gradient(m, T(u_n), Fd)
        q, s, S, U = h.zero_state(n)
        Pbar, dPdF, rnorm, status = h.outputs(n)
        for _ in range(12):
            rv.rve_rom_eval_batch(h, Fd, q, s, S, U, Pbar, dPdF, rnorm, status, precision='fp64')
        R = torch.empty(m.n_dof, dtype=torch.float64, device='cuda')
        Kv = torch.empty(m.nnz, dtype=torch.float64, device='cuda')
        rv.macro_assemble(m, Pbar, dPdF, R, Kv)
        K = sp.csr_matrix((Kv.cpu().numpy(), col, rp), shape=(m.n_dof, m.n_dof))
        gPs = adjoint.reaction_cotangents(prob, K)          # host macro adjoint solve
        e = R.cpu().numpy()[prob.react_dofs].sum() - target[k]
        gF = torch.empty(n, 4, dtype=torch.float64, device='cuda')
        st = torch.empty(n, dtype=torch.int32, device='cuda')
        rv.rve_rom_adjoint(h, Fd, q, T(2.0 * e * gPs.reshape(n, 4)), gF, grad, st)
    torch.cuda.synchronize()
    got = grad.cpu().numpy()[0]
    assert np.abs(got - grad_o).max() <= 1e-8 * np.abs(grad_o).max()
    hh = 1e-6
    for ph in range(2):
        for kk in range(2):
            mp, mm = orom.moduli.copy(), orom.moduli.copy()
            mp[ph, kk] += hh
            mm[ph, kk] -= hh
            Lp = sum((st_[0] - t) ** 2 for st_, t in zip(adjoint.driver_steps(prob, orom.with_moduli(mp), ns, 1e-12), target))
            Lm = sum((st_[0] - t) ** 2 for st_, t in zip(adjoint.driver_steps(prob, orom.with_moduli(mm), ns, 1e-12), target))
            assert abs((Lp - Lm) / (2 * hh) - got[ph, kk]) <= 1e-6 * np.abs(got).max()
