"""Macro level: total-Lagrangian Q4/hex8 elements, the discrete macro
residual R = sum_alpha B_alpha^T Sigma_alpha - F_ext (Sec. 2, Eq. 6, written
here with the first Piola-Kirchhoff stress Pbar), its consistent stiffness
from dPbar/dFbar, and the monolithic and staggered Newton drivers
(Sec. 3.2.3; the flowchart of Sec. 4 is not recoverable, so the iteration
order is read as: evaluate all points -> assemble -> check -> solve -> update,
with the micro update folded into the next evaluation).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Convergence (a reading; the paper gives no norms): max|R_free| <=
tol * max(1, max|R_prescribed|) and max_alpha max|r_alpha| <= tol * mu_matrix * V0.
"""
import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from synthetic import meshes

from . import reduced

_G1 = 1.0 / np.sqrt(3.0)


def _ref_corners(d):
    if d == 2:
        return np.array([[-1, -1], [1, -1], [1, 1], [-1, 1]], dtype=float)
    return np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                     [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=float)


class MacroMesh:
    """Isoparametric Q4 (d=2) / hex8 (d=3) mesh with 2^d Gauss points per
    element.  Integration point alpha = e * 2^d + gp."""

    def __init__(self, X, conn):
        self.X = np.asarray(X, dtype=float)
        self.conn = np.asarray(conn, dtype=np.int64)
        self.d = self.X.shape[1]
        self.nen = 2 ** self.d
        self.n_el = len(self.conn)
        self.n_nodes = len(self.X)
        self.ngp = 2 ** self.d
        self.n_ip = self.n_el * self.ngp
        d = self.d
        s = _ref_corners(d)
        gps = np.array(list(itertools.product([-_G1, _G1], repeat=d)))[:, ::-1]
        dNdxi = np.zeros((len(gps), self.nen, d))
        for q, xi in enumerate(gps):
            for a in range(self.nen):
                for k in range(d):
                    v = s[a, k] / 2.0
                    for m in range(d):
                        if m != k:
                            v *= (1.0 + xi[m] * s[a, m]) / 2.0
                    dNdxi[q, a, k] = v
        Xe = self.X[self.conn]                                # [ne, nen, d]
        Jac = np.einsum('eaI,qak->eqIk', Xe, dNdxi)           # dX_I/dxi_k
        Jinv = np.linalg.inv(Jac)
        detJ = np.linalg.det(Jac)
        if np.any(detJ <= 0):
            raise ValueError("inverted macro element")
        self.dN = np.einsum('qak,eqkI->eqaI', dNdxi, Jinv).reshape(self.n_ip, self.nen, d)
        self.wJ0 = detJ.reshape(self.n_ip)
        self.ip_nodes = np.repeat(self.conn, self.ngp, axis=0)

    def gradient(self, u):
        """Fbar at every integration point from nodal displacements u [nn, d]."""
        ue = u[self.ip_nodes]                                 # [nip, nen, d]
        return np.eye(self.d)[None] + np.einsum('pai,paJ->piJ', ue, self.dN)

    def assemble(self, Pbar, dPdF):
        """Internal force R [nn*d] and stiffness K (sparse) from Pbar
        [nip, d, d] and dPdF [nip, g, g]."""
        d, nen = self.d, self.nen
        Re = np.einsum('p,piJ,paJ->pai', self.wJ0, Pbar, self.dN)
        dofs = (self.ip_nodes[:, :, None] * d + np.arange(d)[None, None, :]).reshape(self.n_ip, nen * d)
        R = np.zeros(self.n_nodes * d)
        np.add.at(R, dofs.ravel(), Re.reshape(-1))
        C = dPdF.reshape(self.n_ip, d, d, d, d)
        Ke = np.einsum('p,paJ,piJkL,pbL->paibk', self.wJ0, self.dN, C, self.dN).reshape(self.n_ip, nen * d, nen * d)
        rows = np.repeat(dofs[:, :, None], nen * d, axis=2)
        cols = np.repeat(dofs[:, None, :], nen * d, axis=1)
        K = sp.csr_matrix((Ke.ravel(), (rows.ravel(), cols.ravel())), shape=(len(R), len(R)))
        return R, K


def rect_mesh(nx, ny, Lx=1.0, Ly=1.0):
    return MacroMesh(*meshes.rect(nx, ny, Lx, Ly))


def box_mesh(nx, ny, nz, Lx, Ly, Lz):
    return MacroMesh(*meshes.box(nx, ny, nz, Lx, Ly, Lz))


def plate_with_hole_mesh(nr, nt, half=1.0, radius=0.2):
    return MacroMesh(*meshes.plate_with_hole(nr, nt, half, radius))


class Problem:
    """Mesh + prescribed DOFs.  presc(lam) gives the prescribed values at load
    factor lam; `react` selects the DOFs whose internal force is summed into
    the reaction."""

    def __init__(self, mesh, presc_dofs, presc_vals, react_dofs):
        self.mesh = mesh
        self.presc_dofs = np.asarray(presc_dofs, dtype=np.int64)
        self.presc_vals = np.asarray(presc_vals, dtype=float)
        self.react_dofs = np.asarray(react_dofs, dtype=np.int64)
        nd = mesh.n_nodes * mesh.d
        mask = np.ones(nd, dtype=bool)
        mask[self.presc_dofs] = False
        self.free = np.nonzero(mask)[0]


def uniaxial_problem(mesh, strain):
    """Left edge u_x = 0, bottom edge u_y = 0, right edge u_x = strain * L."""
    X = mesh.X
    L = X[:, 0].max()
    left = np.nonzero(np.isclose(X[:, 0], 0.0))[0]
    bottom = np.nonzero(np.isclose(X[:, 1], 0.0))[0]
    right = np.nonzero(np.isclose(X[:, 0], L))[0]
    dofs = list(left * 2) + list(bottom * 2 + 1) + list(right * 2)
    vals = [0.0] * (len(left) + len(bottom)) + [strain * L] * len(right)
    return Problem(mesh, dofs, vals, right * 2)


def driver(problem, roms, types, n_steps, scheme='monolithic', tol=1e-10, maxit=30,
           micro_tol=None, keep_steps=False):
    """Load-stepped Newton.  Returns dict(u, reactions[n_steps], iters, hist,
    state, last evaluation list).  With keep_steps the converged u, reaction, K and q of every step are kept."""
    mesh = problem.mesh
    d, nip = mesh.d, mesh.n_ip
    mu_m = roms[0].moduli[0, 0]
    state = [reduced.zero_state(roms[types[a]]) for a in range(nip)]
    from . import rve as rvemod
    for a in range(nip):
        state[a]['Uprev'] = rvemod.to_voigt(np.eye(d))
    u = np.zeros((mesh.n_nodes, d))
    reactions, iters, hist, steps = [], [], [], []
    for n in range(1, n_steps + 1):
        lam = n / n_steps
        uf = u.reshape(-1)
        uf[problem.presc_dofs] = lam * problem.presc_vals
        for it in range(maxit + 1):
            Fbar = mesh.gradient(u)
            if scheme == 'staggered':
                outs = []
                for a in range(nip):
                    o, _ = reduced.converge_point(roms[types[a]], Fbar[a], q0=state[a]['q'],
                                                  tol=micro_tol)
                    outs.append(o)
            else:
                outs = [reduced.eval_point(roms[types[a]], Fbar[a], **state[a]) for a in range(nip)]
            if any(o['status'] != reduced.OK for o in outs):
                raise RuntimeError("micro evaluation failed")
            for a in range(nip):
                state[a] = dict(q=outs[a]['q'], s=outs[a]['s'], S=outs[a]['S'], Uprev=outs[a]['Uprev'])
            Pbar = np.array([o['Pbar'] for o in outs])
            dPdF = np.array([o['dPdF'] for o in outs])
            rmax = max(o['rnorm'] for o in outs)
            R, K = mesh.assemble(Pbar, dPdF)
            Rf = R[problem.free]
            Rp = R[problem.presc_dofs]
            hist.append((n, it, np.max(np.abs(Rf)), rmax))
            if (np.max(np.abs(Rf)) <= tol * max(1.0, np.max(np.abs(Rp)))
                    and rmax <= tol * mu_m * roms[0].V0):
                break
            if it == maxit:
                raise RuntimeError("macro Newton did not converge")
            Kff = K[problem.free][:, problem.free].tocsc()
            du = spla.spsolve(Kff, -Rf)
            uf = u.reshape(-1)
            uf[problem.free] += du
        reactions.append(R[problem.react_dofs].sum())
        iters.append(it)
        if keep_steps:
            steps.append(dict(u=u.copy(), reaction=reactions[-1], K=K.copy(),
                              q=[o['q'].copy() for o in outs]))
    return dict(u=u, reactions=np.array(reactions), iters=iters, hist=hist, state=state,
                outs=outs, K=K, R=R, steps=steps)
