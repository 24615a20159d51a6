"""Pins of the oracle's micro law and polar decomposition against closed
forms, invariants and finite differences (independent of the formula code)."""
import numpy as np
import pytest

from oracle import law, polar

MU, KA = law.mu_kappa_from_E_nu(1.0, 0.3)


def rand_F(rng, d, scale=0.2):
    return np.eye(d) + scale * rng.standard_normal((d, d))


def test_moduli_textbook():
    # Lame's first parameter from (E, nu) by the independent textbook formula
    E, nu = 1.0, 0.3
    lam_hooke = E * nu / ((1 + nu) * (1 - 2 * nu))
    assert abs(law.lam_from(MU, KA) - lam_hooke) < 1e-15
    assert abs(MU - 1.0 / 2.6) < 1e-15 and abs(KA - 1.0 / 1.2) < 1e-15


@pytest.mark.parametrize('d', [2, 3])
def test_stress_free_reference(d):
    assert np.abs(law.stress(np.eye(d), MU, KA)).max() == 0.0


def test_uniaxial_plane_strain_special_case():
    # F = diag(s, 1): J = s, F^-T = diag(1/s, 1); the energy reduces to
    # W(s) = mu/2 (s^2 - 1 - 2 ln s) + lam/2 ln^2 s whose s-derivative is
    # P11 = mu (s - 1/s) + lam ln(s)/s, and P22 = lam ln s, P12 = P21 = 0.
    lam = KA - 2 * MU / 3
    for s in (0.8, 1.1, 1.5):
        P = law.stress(np.diag([s, 1.0]), MU, KA)
        assert abs(P[0, 0] - (MU * (s - 1 / s) + lam * np.log(s) / s)) < 1e-15
        assert abs(P[1, 1] - lam * np.log(s)) < 1e-15
        assert P[0, 1] == 0 and P[1, 0] == 0


@pytest.mark.parametrize('d', [2, 3])
def test_stress_is_energy_gradient(d):
    rng = np.random.default_rng(1)
    F = rand_F(rng, d)
    P = law.stress(F, MU, KA)
    h = 1e-6
    fd = np.zeros((d, d))
    for i in range(d):
        for j in range(d):
            Fp, Fm = F.copy(), F.copy()
            Fp[i, j] += h
            Fm[i, j] -= h
            fd[i, j] = (law.energy(Fp, MU, KA) - law.energy(Fm, MU, KA)) / (2 * h)
    assert np.abs(fd - P).max() <= 1e-8 * np.abs(P).max()


@pytest.mark.parametrize('d', [2, 3])
def test_tangent_is_stress_derivative(d):
    rng = np.random.default_rng(2)
    F = rand_F(rng, d)
    A = law.tangent(F, MU, KA)
    h = 1e-6
    fd = np.zeros_like(A)
    for k in range(d):
        for L in range(d):
            Fp, Fm = F.copy(), F.copy()
            Fp[k, L] += h
            Fm[k, L] -= h
            fd[:, :, k, L] = (law.stress(Fp, MU, KA) - law.stress(Fm, MU, KA)) / (2 * h)
    assert np.abs(fd - A).max() <= 1e-7 * np.abs(A).max()
    # major symmetry of a hyperelastic tangent
    g = d * d
    Am = A.reshape(g, g)
    assert np.abs(Am - Am.T).max() < 1e-14


@pytest.mark.parametrize('d', [2, 3])
def test_small_strain_limit_is_hooke(d):
    # A(I) is the isotropic elasticity tensor lam d_iJ d_kL + mu (d_ik d_JL + d_iL d_Jk)
    lam = law.lam_from(MU, KA)
    I = np.eye(d)
    C = lam * np.einsum('iJ,kL->iJkL', I, I) + MU * (np.einsum('ik,JL->iJkL', I, I)
                                                      + np.einsum('iL,Jk->iJkL', I, I))
    assert np.abs(law.tangent(np.eye(d), MU, KA) - C).max() < 1e-15
    eps = 1e-7 * np.array([[1.0, 0.3, 0.1], [0.3, -0.5, 0.2], [0.1, 0.2, 0.7]])[:d, :d]
    P = law.stress(np.eye(d) + eps, MU, KA)
    hooke = lam * np.trace(eps) * I + 2 * MU * eps
    assert np.abs(P - hooke).max() < 1e-12


@pytest.mark.parametrize('d', [2, 3])
def test_objectivity(d):
    rng = np.random.default_rng(3)
    F = rand_F(rng, d)
    import synthetic as syn
    Q = syn.random_rotation(syn.rng(7), d, 3.0)
    assert np.abs(law.stress(Q @ F, MU, KA) - Q @ law.stress(F, MU, KA)).max() < 1e-14


def test_plane_strain_is_3d_block():
    rng = np.random.default_rng(4)
    F2 = rand_F(rng, 2)
    F3 = np.eye(3)
    F3[:2, :2] = F2
    assert np.abs(law.stress(F3, MU, KA)[:2, :2] - law.stress(F2, MU, KA)).max() < 1e-15
    assert np.abs(law.tangent(F3, MU, KA)[:2, :2, :2, :2] - law.tangent(F2, MU, KA)).max() < 1e-14


def test_moduli_derivatives():
    rng = np.random.default_rng(5)
    F = rand_F(rng, 3)
    dmu, dka = law.stress_dmu_dkappa(F)
    h = 1e-6
    assert np.abs((law.stress(F, MU + h, KA) - law.stress(F, MU - h, KA)) / (2 * h) - dmu).max() < 1e-8
    assert np.abs((law.stress(F, MU, KA + h) - law.stress(F, MU, KA - h)) / (2 * h) - dka).max() < 1e-8


@pytest.mark.parametrize('d', [2, 3])
def test_polar_decomposition(d):
    rng = np.random.default_rng(6)
    for _ in range(5):
        F = rand_F(rng, d, 0.3)
        R, U = polar.polar(F)
        assert np.abs(R @ R.T - np.eye(d)).max() < 1e-14
        assert abs(np.linalg.det(R) - 1) < 1e-14
        assert np.abs(U - U.T).max() == 0.0
        assert np.linalg.eigvalsh(U).min() > 0
        assert np.abs(R @ U - F).max() < 1e-14


def test_polar_2d_matches_3d_embedding():
    rng = np.random.default_rng(8)
    F2 = rand_F(rng, 2, 0.3)
    F3 = np.eye(3)
    F3[:2, :2] = F2
    R2, U2 = polar.polar(F2)
    R3, U3 = polar.polar(F3)
    assert np.abs(R3[:2, :2] - R2).max() < 1e-14 and np.abs(U3[:2, :2] - U2).max() < 1e-14


@pytest.mark.parametrize('d', [2, 3])
def test_polar_derivative_fd(d):
    rng = np.random.default_rng(9)
    F = rand_F(rng, d, 0.3)
    R, U = polar.polar(F)
    h = 1e-6
    for _ in range(3):
        dF = rng.standard_normal((d, d))
        dR, dU = polar.polar_derivative(R, U, dF)
        Rp, Up = polar.polar(F + h * dF)
        Rm, Um = polar.polar(F - h * dF)
        assert np.abs((Rp - Rm) / (2 * h) - dR).max() < 1e-8
        assert np.abs((Up - Um) / (2 * h) - dU).max() < 1e-8
