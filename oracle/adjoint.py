"""Implicit-function adjoint of the converged reduced RVE equilibrium.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper has no adjoint; this is the differentiation through the converged
hyper-reduced micro problem r(q*, U, theta) = 0 (Sec. 3.2.3 notation):
    dq*/dtheta = -K^-1 dr/dtheta,   dr/dtheta = sum_i w_i B_i^T dP_i/dtheta
    dPbar_U/dtheta = (1/V0) [sum_i w_i dP_i/dtheta + K_qF^T dq*/dtheta]
so for a cotangent gP on Pbar = R Pbar_U (R independent of theta):
    gPU = R^T gP,   z = K^-1 K_qF gPU,
    g_theta = (1/V0) sum_i w_i < gPU - B_i z , dP_i/dtheta >
with theta = (mu, kappa) of the phase of ECM point i.  The cotangent on Fbar
is gF = (dPbar/dFbar)^T gP with the condensed consistent tangent.

Macro level (reaction-force loss): at a converged macro state R_free = 0, the
derivative of c^T R_int (c selects the reaction DOFs) is
    (c + psi)^T dR_int/dtheta,  psi_free = -K_ff^-T K_pf^T c_p,  psi_p = 0,
and dR_int/dtheta = sum_alpha wJ0 dN^T dPbar_alpha/dtheta, so each point
receives the cotangent gP_alpha[i,J] = wJ0 sum_a (c+psi)[a,i] dN_a,J.
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import law, reduced, polar as pol


def point_adjoint(rom, Fbar, q, gP):
    """Return (gF [g], gtheta [n_phase, 2]) at the (converged) state q."""
    d, g = rom.d, rom.g
    st = reduced.zero_state(rom)
    R, U = pol.polar(Fbar)
    from . import rve as rvemod
    o = reduced.eval_point(rom, Fbar, q, st['s'], st['S'], rvemod.to_voigt(U))
    if o['status'] != reduced.OK:
        raise RuntimeError("adjoint at an invalid state")
    gP = np.asarray(gP, dtype=float).reshape(d, d)
    gF = o['dPdF'].T @ gP.ravel()
    gPU = (R.T @ gP).ravel()
    z = np.linalg.solve(o['K'], o['KqF'] @ gPU)
    F = (U.reshape(1, g) + np.einsum('icj,j->ic', rom.B, q)).reshape(rom.m, d, d)
    dmu, dka = law.stress_dmu_dkappa(F)
    v = gPU[None, :] - np.einsum('icj,j->ic', rom.B, z)          # [m, g]
    gth = np.zeros((rom.moduli.shape[0], 2))
    cmu = rom.w * np.einsum('ic,ic->i', v, dmu.reshape(rom.m, g)) / rom.V0
    cka = rom.w * np.einsum('ic,ic->i', v, dka.reshape(rom.m, g)) / rom.V0
    np.add.at(gth[:, 0], rom.phase, cmu)
    np.add.at(gth[:, 1], rom.phase, cka)
    return gF, gth


def reaction_cotangents(problem, K):
    """Per-point cotangents gP (nip, d, d) of the reaction c^T R_int."""
    mesh = problem.mesh
    d = mesh.d
    nd = mesh.n_nodes * d
    c = np.zeros(nd)
    c[problem.react_dofs] = 1.0
    Kc = K.tocsc()
    Kff = Kc[problem.free][:, problem.free]
    Kpf = Kc[problem.presc_dofs][:, problem.free]
    psi = np.zeros(nd)
    psi[problem.free] = -spla.spsolve(Kff.T.tocsc(), Kpf.T @ c[problem.presc_dofs])
    v = (c + psi).reshape(mesh.n_nodes, d)[mesh.ip_nodes]          # [nip, nen, d]
    return np.einsum('p,pai,paJ->piJ', mesh.wJ0, v, mesh.dN)


def reaction_loss_and_grad(problem, rom, n_steps, target, tol=1e-11):
    """Loss sum_n (reaction_n - target_n)^2 along the load path and its
    gradient with respect to rom.moduli [n_phase, 2]."""
    nip = problem.mesh.n_ip
    types = np.zeros(nip, dtype=np.int64)
    mesh = problem.mesh
    d = mesh.d
    u = np.zeros((mesh.n_nodes, d))
    res = driver_steps(problem, rom, n_steps, tol)
    L = 0.0
    grad = np.zeros_like(rom.moduli)
    for n, (reac, u_n, K_n, qs) in enumerate(res):
        e = reac - target[n]
        L += e * e
        gPs = reaction_cotangents(problem, K_n)
        Fbar = mesh.gradient(u_n)
        for a in range(nip):
            _, gth = point_adjoint(rom, Fbar[a], qs[a], 2.0 * e * gPs[a])
            grad += gth
    return L, grad


def driver_steps(problem, rom, n_steps, tol):
    """Converged (u, reaction, K, q per point) at every load step, from the
    monolithic driver of oracle.macro run one step at a time."""
    from . import macro
    out = []
    r = macro.driver(problem, [rom], np.zeros(problem.mesh.n_ip, dtype=np.int64), n_steps,
                     tol=tol, keep_steps=True)
    for n in range(n_steps):
        st = r['steps'][n]
        out.append((st['reaction'], st['u'], st['K'], st['q']))
    return out
