"""Pins of the full-order periodic RVE oracle (Sec. 2, Eqs. 1-8)."""
import numpy as np
import pytest

from oracle import law, rve

MU, KA = law.mu_kappa_from_E_nu(1.0, 0.3)
MOD = [[MU, KA], [10 * MU, 10 * KA]]


def model(d, n, homogeneous=False, vf=0.2):
    ph = rve.phases_single_inclusion(d, n, vf)
    mods = [MOD[0], MOD[0]] if homogeneous else MOD
    return rve.PeriodicRVE(d, n, ph, mods)


def F2():
    return np.array([[1.07, 0.03], [-0.02, 0.96]])


def F3():
    return np.array([[1.05, 0.02, -0.01], [0.01, 0.97, 0.03], [0.0, -0.02, 1.02]])


@pytest.mark.parametrize('d,n', [(2, 6), (3, 3)])
def test_average_of_periodic_gradient_is_zero(d, n):
    # Eq. 3: the volume average of grad w vanishes for periodic w, so <F> = Fbar
    m = model(d, n)
    w = np.random.default_rng(0).standard_normal(m.n_dof)
    gw = (m.G @ w).reshape(m.n_ip, d * d)
    assert np.abs(m.ip_weight @ gw).max() < 1e-12
    assert abs(m.ip_weight.sum() - m.V0) < 1e-14


@pytest.mark.parametrize('d,n,Fb', [(2, 6, F2()), (3, 3, F3())])
def test_homogeneous_rve_reproduces_law(d, n, Fb):
    m = model(d, n, homogeneous=True)
    w, Pbar, Cbar, it = m.solve(Fb)
    assert np.abs(w).max() < 1e-13
    assert np.abs(Pbar - law.stress(Fb, MU, KA)).max() < 1e-14
    assert np.abs(Cbar - law.tangent(Fb, MU, KA).reshape(d * d, d * d)).max() < 1e-13


def _avg_energy(m, Fb, w):
    F = m.F_at_ips(Fb, w)
    return m.ip_weight @ law.energy(F, m.ip_mu, m.ip_kappa) / m.V0


@pytest.mark.parametrize('d,n,Fb', [(2, 8, F2()), (3, 3, F3())])
def test_hill_mandel_and_condensed_tangent(d, n, Fb):
    m = model(d, n)
    w, Pbar, Cbar, _ = m.solve(Fb)
    h = 1e-6
    g = d * d
    fdP = np.zeros(g)
    fdC = np.zeros((g, g))
    for c in range(g):
        dF = np.zeros(g)
        dF[c] = h
        dF = dF.reshape(d, d)
        wp, Pp, _, _ = m.solve(Fb + dF, w0=w)
        wm, Pm, _, _ = m.solve(Fb - dF, w0=w)
        # macro stress is the derivative of the averaged energy (Hill-Mandel)
        fdP[c] = (_avg_energy(m, Fb + dF, wp) - _avg_energy(m, Fb - dF, wm)) / (2 * h)
        fdC[:, c] = ((Pp - Pm) / (2 * h)).ravel()
    assert np.abs(fdP - Pbar.ravel()).max() < 1e-8 * np.abs(Pbar).max()
    assert np.abs(fdC - Cbar).max() < 1e-6 * np.abs(Cbar).max()
    # power equivalence for an arbitrary macro rate with the equilibrium w
    dF = np.random.default_rng(1).standard_normal((d, d))
    F = m.F_at_ips(Fb, w)
    P = law.stress(F, m.ip_mu, m.ip_kappa)
    dw = np.random.default_rng(2).standard_normal(m.n_dof) * 1e-3
    micro = m.ip_weight @ np.einsum('piJ,piJ->p', P, dF[None] + (m.G @ dw).reshape(m.n_ip, d, d))
    assert abs(micro - m.V0 * np.sum(Pbar * dF)) < 1e-10


@pytest.mark.parametrize('d,n,Fb', [(2, 8, F2()), (3, 3, F3())])
def test_macro_objectivity(d, n, Fb):
    import synthetic as syn
    m = model(d, n)
    Q = syn.random_rotation(syn.rng(11), d, 1.0)
    _, P1, _, _ = m.solve(Fb)
    _, P2, _, _ = m.solve(Q @ Fb)
    assert np.abs(P2 - Q @ P1).max() < 1e-12


def test_voigt_reuss_bounds():
    # at Fbar = I the effective tangent is bracketed by the phase averages
    d, n = 2, 12
    m = model(d, n)
    _, _, C, _ = m.solve(np.eye(d))
    vf = m.phase.mean()
    Cm = law.tangent(np.eye(d), *MOD[0]).reshape(4, 4)
    Ci = law.tangent(np.eye(d), *MOD[1]).reshape(4, 4)
    E = rve.voigt_map(d)
    S = E.T @ E                     # metric of tensor components in Voigt space
    Cv = E.T @ ((1 - vf) * Cm + vf * Ci) @ E
    Ce = E.T @ C @ E
    Pinv = lambda M: np.linalg.inv(M)
    Cr = np.linalg.inv((1 - vf) * Pinv(E.T @ Cm @ E) + vf * Pinv(E.T @ Ci @ E))
    assert np.linalg.eigvalsh(Cv - Ce).min() > -1e-12
    assert np.linalg.eigvalsh(Ce - Cr).min() > -1e-12
    assert np.linalg.eigvalsh(S).min() > 0


def test_mesh_convergence():
    Fb = F2()
    P = {}
    for n in (8, 16, 32):
        _, P[n], _, _ = model(2, n).solve(Fb)
    e8 = np.abs(P[8] - P[32]).max()
    e16 = np.abs(P[16] - P[32]).max()
    assert e16 < e8
