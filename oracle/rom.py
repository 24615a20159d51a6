"""Offline stage: training snapshots, POD with elastic/inelastic split, ROM
training runs with full integration, and the empirical cubature method.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

  snapshots     converged full-order fluctuations along training stretch paths
                (stretch only, Sec. 3.2.2: no rotations are trained)
  pod_basis     Eq. SVD_displacement / Eq. snapshots_displacement: Phi_el
                spans the elastic range, Phi_inel are the leading left
                singular vectors of the snapshots with their Phi_el part
                removed; Phi = [Phi_el Phi_inel]
  ecm_training  per-integration-point integrands f~^{kg} = [B_g^T P_g ; P_g]
                along the training paths with full integration, and the
                training matrix x_f of Sec. 3.3 (rows f~^{kg}_i - f~^k_i/V0)
  ecm_greedy    Box 1 (greedy non-negative point selection) on
                J = [lambda 1]^T, b = [0 V0]^T, lambda = leading m~-1 left
                singular vectors of x_f^T (Eq. SVDlambda)

Readings where the paper is garbled or silent:
  * the elastic snapshots of a hyperelastic RVE are the linearized responses
    to the n_sigma unit macro strains at Fbar = I;
  * Box 1 starts from r = b but its step 7 prints r = J w - b; the residual
    is taken as r = b - J_z w so that step 1 picks the column most aligned
    with what is still missing; ties go to the lowest index;
  * x_f rows are scaled blockwise (mode block, stress block) to unit
    Frobenius norm before the SVD; the stress block holds all g components
    of P (the macro stress of this formulation is the unsymmetric P).
"""
import numpy as np
import scipy.optimize as spo

from . import reduced


def snapshots(model, paths):
    """paths [n_paths, n_steps, d, d] -> X (n_dof x n_paths*n_steps)."""
    cols = []
    for p in range(paths.shape[0]):
        w = None
        for k in range(paths.shape[1]):
            w, _, _, _ = model.solve(paths[p, k], w0=w)
            cols.append(w.copy())
    return np.array(cols).T


def pod_basis(model, X, n_modes):
    Wel = model.linear_responses()
    Phi_el = np.linalg.svd(Wel, full_matrices=False)[0]
    Xmod = X - Phi_el @ (Phi_el.T @ X)
    Uin = np.linalg.svd(Xmod, full_matrices=False)[0]
    Phi = np.hstack([Phi_el, Uin[:, :n_modes - Phi_el.shape[1]]])
    return Phi


def full_integration_rom(model, Phi):
    """ROM with all micro integration points and their Gauss weights."""
    g, n = model.g, Phi.shape[1]
    B = np.asarray(model.G @ Phi).reshape(model.n_ip, g, n)
    return reduced.Rom(B, model.ip_weight, model.ip_phase, model.moduli, model.V0)


def ecm_training(model, Phi, paths, tol=None):
    """Run the fully integrated ROM along the paths (micro converged at every
    step) and return the list of per-point integrand arrays [m, n + g]."""
    rom = full_integration_rom(model, Phi)
    fk = []
    for p in range(paths.shape[0]):
        q = None
        for k in range(paths.shape[1]):
            o, _ = reduced.converge_point(rom, paths[p, k], q0=q, tol=tol)
            if o['status'] != reduced.OK:
                raise RuntimeError("ROM training run failed")
            q = o['q']
            F = rom.B @ q + o['U'].reshape(1, -1)
            from . import law
            mu = rom.moduli[rom.phase, 0]
            ka = rom.moduli[rom.phase, 1]
            P = law.stress(F.reshape(rom.m, rom.d, rom.d), mu, ka).reshape(rom.m, rom.g)
            fk.append(np.hstack([np.einsum('pcj,pc->pj', rom.B, P), P]))
    return fk


def training_matrix(fk, weights, V0, n_modes):
    rows = []
    for f in fk:
        fint = weights @ f                       # sum_g w_g f~^{kg}
        rows.append((f - fint[None, :] / V0).T)  # [n_t, m]
    xf = np.vstack(rows)
    n_t = fk[0].shape[1]
    blk = np.tile(np.arange(n_t) < n_modes, len(fk))
    for sel in (blk, ~blk):
        nrm = np.linalg.norm(xf[sel])
        if nrm > 0:
            xf[sel] /= nrm
    return xf


def ecm_greedy(J, b, m_target):
    m = J.shape[1]
    norms = np.linalg.norm(J, axis=0)
    available = np.ones(m, dtype=bool)
    z, w = [], np.zeros(0)
    r = b.copy()
    while len(z) < m_target and available.any():
        score = (J.T @ r) / norms
        score[~available] = -np.inf
        k = int(np.argmax(score))
        z.append(k)
        available[k] = False
        w = np.linalg.lstsq(J[:, z], b, rcond=None)[0]
        if np.any(w < 0):
            w = spo.nnls(J[:, z], b)[0]
            keep = w > 0
            z = [z[t] for t in range(len(z)) if keep[t]]
            w = w[keep]
        r = b - J[:, z] @ w
    return np.array(z, dtype=np.int64), w


def ecm(xf, V0, m_target):
    Vt = np.linalg.svd(xf, full_matrices=False)[2]     # x_f = U s V^T, x_f^T = V s U^T
    lam = Vt[:m_target - 1].T                          # m x (m~ - 1)
    m = lam.shape[0]
    J = np.vstack([lam.T, np.ones((1, m))])
    b = np.zeros(m_target)
    b[-1] = V0
    return ecm_greedy(J, b, m_target)


def hyper_rom(model, Phi, z, w):
    full = full_integration_rom(model, Phi)
    return reduced.Rom(full.B[z], w, full.phase[z], model.moduli, model.V0)


def save_rom(path, rom, **meta):
    np.savez_compressed(path, B=rom.B, w=rom.w, phase=rom.phase.astype(np.int32),
                        moduli=rom.moduli, V0=rom.V0, **meta)
