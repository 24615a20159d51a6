"""Pins of the hyper-reduced evaluation (Sec. 3.2.2-3.2.3), the macro element
and Newton drivers (Eq. 6) and the implicit adjoint, on the committed
16x16 / 12-mode / 60-point ROM."""
import numpy as np
import pytest

import synthetic as syn
from oracle import law, macro, reduced, adjoint, polar, rve
from conftest import rom_path


@pytest.fixture(scope='module')
def rom1():
    return reduced.Rom.load(rom_path('c1'))


def test_rom_file_invariants(rom1):
    assert rom1.B.shape == (60, 4, 12)
    assert abs(rom1.w.sum() - rom1.V0) < 1e-12 and np.all(rom1.w > 0)


def test_condensed_tangent_matches_fd_of_converged_stress(rom1):
    Fb = syn.fbar_batch(21, 2, 1, 0.1, 0.3)[0]
    o, _ = reduced.converge_point(rom1, Fb)
    h = 1e-6
    fd = np.zeros((4, 4))
    for c in range(4):
        dF = np.zeros(4)
        dF[c] = h
        op, _ = reduced.converge_point(rom1, Fb + dF.reshape(2, 2), q0=o['q'])
        om, _ = reduced.converge_point(rom1, Fb - dF.reshape(2, 2), q0=o['q'])
        fd[:, c] = ((op['Pbar'] - om['Pbar']) / (2 * h)).ravel()
    assert np.abs(fd - o['dPdF']).max() < 1e-6 * np.abs(o['dPdF']).max()


def test_algorithmic_stress_is_first_order_prediction(rom1):
    # Sigma_alg = Sigma - dSigma/dq K^-1 r predicts the stress after the
    # pending micro correction to second order in the perturbation
    Fb = syn.fbar_batch(22, 2, 1, 0.1, 0.0)[0]
    oc, _ = reduced.converge_point(rom1, Fb)
    R, U = polar.polar(Fb)
    dq = syn.perturbation(5, rom1.n, 1e-3 * np.abs(oc['q']).max())
    z = reduced.zero_state(rom1)
    o = reduced.eval_point(rom1, Fb, oc['q'] + dq, z['s'], z['S'], rve.to_voigt(U))
    PU = (reduced.reduced_system(rom1, U, oc['q'] + dq)[1] / rom1.V0).reshape(2, 2)
    err_alg = np.abs(o['Palg'] - oc['Palg']).max()
    err_raw = np.abs(PU - oc['Palg']).max()
    assert err_alg < 1e-3 * err_raw


def test_reduced_objectivity(rom1):
    Fb = syn.fbar_batch(23, 2, 1, 0.1, 0.0)[0]
    Q = syn.random_rotation(syn.rng(3), 2, 2.0)
    o1, _ = reduced.converge_point(rom1, Fb)
    o2, _ = reduced.converge_point(rom1, Q @ Fb)
    assert np.abs(o2['Pbar'] - Q @ o1['Pbar']).max() < 1e-14


def test_monolithic_update_uses_stored_sensitivities(rom1):
    # q <- q - s - S dU is one Newton step of the coupled system: after it,
    # the residual at the new stretch is second order in dU
    Fb = syn.fbar_batch(24, 2, 1, 0.1, 0.0)[0]
    oc, _ = reduced.converge_point(rom1, Fb)
    dU = 1e-4 * np.array([[1.0, 0.5], [0.5, -0.7]])
    o = reduced.eval_point(rom1, Fb + dU, oc['q'], oc['s'], oc['S'], oc['Uprev'])
    o0 = reduced.eval_point(rom1, Fb + dU, oc['q'], 0 * oc['s'], 0 * oc['S'], oc['Uprev'])
    assert o['rnorm'] < 1e-3 * o0['rnorm']


def test_macro_patch_and_stiffness_fd():
    mesh = macro.rect_mesh(3, 2, 1.5, 1.0)
    H = np.array([[0.05, 0.02], [-0.01, 0.03]])
    u = mesh.X @ H.T
    Fb = mesh.gradient(u)
    assert np.abs(Fb - (np.eye(2) + H)[None]).max() < 1e-15
    mu, ka = law.mu_kappa_from_E_nu(1.0, 0.3)
    P = law.stress(Fb, mu, ka)
    R, _ = mesh.assemble(P, law.tangent(Fb, mu, ka).reshape(-1, 4, 4))
    interior = [n for n in range(mesh.n_nodes) if 0 < mesh.X[n, 0] < 1.5 and 0 < mesh.X[n, 1] < 1.0]
    assert np.abs(R.reshape(-1, 2)[interior]).max() < 1e-15
    # total force balance of a homogeneous stress field
    assert np.abs(R.reshape(-1, 2).sum(0)).max() < 1e-14
    rng = np.random.default_rng(0)
    u = 0.02 * rng.standard_normal((mesh.n_nodes, 2))
    Fb = mesh.gradient(u)
    R0, K = mesh.assemble(law.stress(Fb, mu, ka), law.tangent(Fb, mu, ka).reshape(-1, 4, 4))
    K = K.toarray()
    h = 1e-6
    for dof in (0, 5, 11):
        up, um = u.copy().ravel(), u.copy().ravel()
        up[dof] += h
        um[dof] -= h
        Fp, Fm = mesh.gradient(up.reshape(-1, 2)), mesh.gradient(um.reshape(-1, 2))
        Rp, _ = mesh.assemble(law.stress(Fp, mu, ka), law.tangent(Fp, mu, ka).reshape(-1, 4, 4))
        Rm, _ = mesh.assemble(law.stress(Fm, mu, ka), law.tangent(Fm, mu, ka).reshape(-1, 4, 4))
        assert np.abs((Rp - Rm) / (2 * h) - K[:, dof]).max() < 1e-8


def test_hex8_patch():
    mesh = macro.box_mesh(2, 2, 1, 1.0, 1.0, 0.5)
    assert abs(mesh.wJ0.sum() - 0.5) < 1e-14
    H = np.array([[0.05, 0.02, 0.0], [-0.01, 0.03, 0.01], [0.02, 0.0, -0.02]])
    assert np.abs(mesh.gradient(mesh.X @ H.T) - (np.eye(3) + H)[None]).max() < 1e-15


def test_monolithic_equals_staggered_and_converges_quadratically(rom1):
    p = macro.uniaxial_problem(macro.rect_mesh(2, 2), 0.1)
    types = np.zeros(p.mesh.n_ip, dtype=np.int64)
    mono = macro.driver(p, [rom1], types, 5)
    stag = macro.driver(p, [rom1], types, 5, scheme='staggered')
    assert np.abs(mono['u'] - stag['u']).max() < 1e-12
    assert np.abs(mono['reactions'] - stag['reactions']).max() < 1e-11
    # quadratic: each residual is far below the square of the previous one
    # (relative to the first residual of the step) once in the asymptotic range
    h = [x for x in mono['hist'] if x[0] == 3]
    r = [x[2] for x in h]
    assert len(r) >= 3 and r[2] < 10 * r[1] ** 2 / r[0] + 1e-14


def test_point_adjoint_matches_fd(rom1):
    Fb = syn.fbar_batch(25, 2, 1, 0.1, 0.3)[0]
    o, _ = reduced.converge_point(rom1, Fb)
    gP = syn.perturbation(9, (2, 2), 1.0)
    gF, gth = adjoint.point_adjoint(rom1, Fb, o['q'], gP)
    assert np.abs(gF - o['dPdF'].T @ gP.ravel()).max() < 1e-14
    h = 1e-6
    for ph in range(2):
        for k in range(2):
            mp, mm = rom1.moduli.copy(), rom1.moduli.copy()
            mp[ph, k] += h
            mm[ph, k] -= h
            op, _ = reduced.converge_point(rom1.with_moduli(mp), Fb, q0=o['q'])
            om, _ = reduced.converge_point(rom1.with_moduli(mm), Fb, q0=o['q'])
            fd = np.sum(gP * (op['Pbar'] - om['Pbar'])) / (2 * h)
            assert abs(fd - gth[ph, k]) < 1e-6 * max(1.0, abs(gth[ph, k]))


def test_reaction_loss_gradient_fd_and_zero_at_target(rom1):
    p = macro.uniaxial_problem(macro.rect_mesh(2, 2), 0.1)
    ns = 3
    g = syn.rng(syn.SEED_BASE + 4)
    scale = 0.8 + 0.4 * g.random((2, 2))
    target_rom = rom1.with_moduli(rom1.moduli * scale)
    target = np.array([s[0] for s in adjoint.driver_steps(p, target_rom, ns, 1e-12)])
    L0, g0 = adjoint.reaction_loss_and_grad(p, target_rom, ns, target)
    assert L0 < 1e-20 and np.abs(g0).max() < 1e-9
    L, grad = adjoint.reaction_loss_and_grad(p, rom1, ns, target)
    h = 1e-6
    for ph in range(2):
        for k in range(2):
            mp, mm = rom1.moduli.copy(), rom1.moduli.copy()
            mp[ph, k] += h
            mm[ph, k] -= h
            Lp = sum((s[0] - t) ** 2 for s, t in zip(adjoint.driver_steps(p, rom1.with_moduli(mp), ns, 1e-12), target))
            Lm = sum((s[0] - t) ** 2 for s, t in zip(adjoint.driver_steps(p, rom1.with_moduli(mm), ns, 1e-12), target))
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - grad[ph, k]) <= 1e-6 * np.abs(grad).max()
