"""Biot and Cauchy outputs of the homogenized response (Sec. 3.2.2, Eqs.
workconjugacy and biotstress; Appendix A), for macro codes that work with
the true stress in an updated-Lagrangian setting.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

With Fbar = R U (polar split) and the homogenized first Piola-Kirchhoff
stress P and its tangent dP/dF:
  Biot stress        T = sym(R^T P)                 (work conjugate to U)
  Biot tangent       C^B[v][w] = dT_v / dU_w for symmetric stretch variations
                     dU = E e_w at fixed R (then dF = R dU and dR = 0)
  Cauchy stress      sigma from T = (J/2)(R^T sigma F^-T + F^-1 sigma R),
                     the linear relation of Eq. biotstress, solved for the
                     symmetric sigma
  Cauchy tangent     dsigma/dD ~ (dsigma/dT) : C^B : dUdot/dD with the
                     approximation dUdot/dD ~ R_ki F_lj of Appendix A (constant
                     rotation over the step), applied to the symmetric part.
Symmetric tensors are stored by their independent tensor components in the
project's order (2D 11, 22, 12; 3D 11, 22, 33, 12, 13, 23).
"""
import numpy as np

from . import polar as pol, rve as rvemod


def _basis(d):
    """Symmetric unit tensors E_v (tensor components: both off-diagonal
    entries 1 for a shear component)."""
    E = rvemod.voigt_map(d)
    return [E[:, v].reshape(d, d) for v in range(E.shape[1])]


def biot_stress(Fbar, P):
    R, _ = pol.polar(Fbar)
    T = R.T @ np.asarray(P).reshape(R.shape)
    return rvemod.to_voigt(0.5 * (T + T.T))


def biot_tangent(Fbar, dPdF):
    d = Fbar.shape[0]
    R, _ = pol.polar(Fbar)
    C = np.zeros((len(_basis(d)), len(_basis(d))))
    for w, Ew in enumerate(_basis(d)):
        dP = (np.asarray(dPdF) @ (R @ Ew).ravel()).reshape(d, d)
        dT = R.T @ dP
        C[:, w] = rvemod.to_voigt(0.5 * (dT + dT.T))
    return C


def _biot_map(Fbar):
    """Matrix L (ns x ns) of the linear map sigma -> T of Eq. biotstress on
    symmetric tensors."""
    d = Fbar.shape[0]
    R, _ = pol.polar(Fbar)
    Fi = np.linalg.inv(Fbar)
    J = np.linalg.det(Fbar)
    B = _basis(d)
    L = np.zeros((len(B), len(B)))
    for w, Ew in enumerate(B):
        T = 0.5 * J * (R.T @ Ew @ Fi.T + Fi @ Ew @ R)
        L[:, w] = rvemod.to_voigt(T)
    return L


def cauchy_stress(Fbar, T):
    return np.linalg.solve(_biot_map(Fbar), np.asarray(T))


def cauchy_tangent(Fbar, CB):
    d = Fbar.shape[0]
    R, _ = pol.polar(Fbar)
    L = _biot_map(Fbar)
    B = _basis(d)
    G = np.zeros((len(B), len(B)))              # sym(R^T D F) for D = E_w
    for w, Ew in enumerate(B):
        X = R.T @ Ew @ Fbar
        G[:, w] = rvemod.to_voigt(0.5 * (X + X.T))
    return np.linalg.solve(L, CB @ G)


def outputs(Fbar, P, dPdF):
    """(T, C^B, sigma, dsigma/dD) of one point."""
    T = biot_stress(Fbar, P)
    CB = biot_tangent(Fbar, dPdF)
    return T, CB, cauchy_stress(Fbar, T), cauchy_tangent(Fbar, CB)
