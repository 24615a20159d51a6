"""Polar decomposition F = R U of the macro deformation gradient and its
derivative (Sec. 3.2.2, Eq. polar_decomp: only the stretch U is imposed on the
RVE; the rotation R is applied to the homogenized response afterwards).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

2D: R is the rotation by theta = atan2(F21 - F12, F11 + F22), U = R^T F.
3D: the recipe of the appendix (commented part of Appendix A): eigen
decomposition of C = F^T F gives U = V sqrt(L) V^T, then R = F U^-1.

Derivative: with dF = dR U + R dU, Omega = R^T dR skew and dU symmetric,
    Omega U + U Omega = R^T dF - dF^T R           (a Sylvester equation)
whose skew solution is  omega = W21 / tr U  in 2D (Omega = omega [[0,-1],[1,0]])
and  (tr U I - U) omega = w  in 3D for the axial vectors omega, w of Omega and
of the right-hand side.  Then dU = R^T dF - Omega U and dR = R Omega.
"""
import numpy as np


def polar(F):
    F = np.asarray(F, dtype=float)
    d = F.shape[-1]
    if d == 2:
        th = np.arctan2(F[1, 0] - F[0, 1], F[0, 0] + F[1, 1])
        c, s = np.cos(th), np.sin(th)
        R = np.array([[c, -s], [s, c]])
        U = R.T @ F
        U = 0.5 * (U + U.T)
        return R, U
    C = F.T @ F
    lam, V = np.linalg.eigh(C)
    U = V @ np.diag(np.sqrt(lam)) @ V.T
    U = 0.5 * (U + U.T)
    Uinv = V @ np.diag(1.0 / np.sqrt(lam)) @ V.T
    R = F @ Uinv
    return R, U


def _axial(W):
    return np.array([W[2, 1], W[0, 2], W[1, 0]])


def _skew(w):
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def polar_derivative(R, U, dF):
    """Return (dR, dU) for a perturbation dF of F = R U."""
    d = U.shape[0]
    X = R.T @ dF
    W = X - X.T
    if d == 2:
        om = W[1, 0] / np.trace(U)
        Om = np.array([[0.0, -om], [om, 0.0]])
    else:
        om = np.linalg.solve(np.trace(U) * np.eye(3) - U, _axial(W))
        Om = _skew(om)
    dU = X - Om @ U
    dU = 0.5 * (dU + dU.T)
    return R @ Om, dU
