"""Compressible Neo-Hooke law, the pointwise micro law of the hot path.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper does not fix a finite-strain micro law for the hyperelastic case, so
the project reads it as the standard compressible Neo-Hooke energy
    W(F) = mu/2 (tr C - d3 - 2 ln J) + lam/2 (ln J)^2,  lam = kappa - 2 mu / 3,
with C = F^T F, J = det F and d3 = 3 (plane strain embeds F in 3D with
F33 = 1, so the in-plane blocks of the 3D expressions are exact).
    P = dW/dF = mu (F - F^-T) + lam ln J F^-T
    A_iJkL = dP_iJ / dF_kL
           = mu d_ik d_JL + lam Finv_Ji Finv_Lk + (mu - lam ln J) Finv_Li Finv_Jk
All arrays are float64; F has shape (..., d, d), moduli broadcast over '...'.
"""
import numpy as np


def lam_from(mu, kappa):
    return kappa - 2.0 * mu / 3.0


def mu_kappa_from_E_nu(E, nu):
    """Shear and bulk modulus of an isotropic solid from Young's modulus and
    Poisson's ratio (textbook relations)."""
    return E / (2.0 * (1.0 + nu)), E / (3.0 * (1.0 - 2.0 * nu))


def energy(F, mu, kappa):
    lam = lam_from(mu, kappa)
    d = F.shape[-1]
    J = np.linalg.det(F)
    trC = np.einsum('...iJ,...iJ->...', F, F) + (3 - d)
    lnJ = np.log(J)
    return 0.5 * mu * (trC - 3.0 - 2.0 * lnJ) + 0.5 * lam * lnJ ** 2


def stress(F, mu, kappa):
    """First Piola-Kirchhoff stress P(F)."""
    mu = np.asarray(mu, dtype=float)[..., None, None]
    lam = lam_from(mu, np.asarray(kappa, dtype=float)[..., None, None])
    Finv = np.linalg.inv(F)
    FinvT = np.swapaxes(Finv, -1, -2)
    lnJ = np.log(np.linalg.det(F))[..., None, None]
    return mu * (F - FinvT) + lam * lnJ * FinvT


def tangent(F, mu, kappa):
    """A_iJkL = dP_iJ/dF_kL, shape (..., d, d, d, d)."""
    d = F.shape[-1]
    mu = np.asarray(mu, dtype=float)[..., None, None, None, None]
    lam = lam_from(mu, np.asarray(kappa, dtype=float)[..., None, None, None, None])
    Finv = np.linalg.inv(F)
    lnJ = np.log(np.linalg.det(F))[..., None, None, None, None]
    I = np.eye(d)
    t1 = np.einsum('ik,JL->iJkL', I, I)
    t2 = np.einsum('...Ji,...Lk->...iJkL', Finv, Finv)
    t3 = np.einsum('...Li,...Jk->...iJkL', Finv, Finv)
    return mu * t1 + lam * t2 + (mu - lam * lnJ) * t3


def stress_dmu_dkappa(F):
    """Partial derivatives of P with respect to the moduli (mu, kappa) at
    fixed F, used by the adjoint:  dP/dmu = F - F^-T - (2/3) ln J F^-T,
    dP/dkappa = ln J F^-T."""
    Finv = np.linalg.inv(F)
    FinvT = np.swapaxes(Finv, -1, -2)
    lnJ = np.log(np.linalg.det(F))[..., None, None]
    return F - FinvT - (2.0 / 3.0) * lnJ * FinvT, lnJ * FinvT
