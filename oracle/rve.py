"""Full-order periodic RVE finite elements (Sec. 2: Eqs. 2-3 homogenization,
Eq. FEM_micro periodic boundary value problem, Eq. 8 micro residual with the
macro stress as reaction to H).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Formulation.  The paper eliminates the "-" boundary nodes with a matrix A that
ties u^- to u^+ and H.  Equivalently (and this is the form used here and by the
ROM), the micro displacement is u = H X + w with a periodic fluctuation w; the
deformation gradient at a micro integration point p is
    F_p = Fbar + grad w (X_p) = Fbar + G_p w,
where G_p (g x n) maps the independent fluctuation DOFs to the g = d^2
components of grad w (row-major flattening c = i*d + J).  Periodicity is built
into the DOF numbering (node index mod n); the fluctuation of node 0 is fixed
to zero to remove the rigid translation.

Homogenization: Pbar = (1/V0) sum_p w_p P(F_p)  (Eq. 2 evaluated by Gauss
quadrature), the micro residual f = G^T diag(w) P, and the condensed tangent
    Cbar = (1/V0) (K_FF - K_wF^T K_ww^-1 K_wF)
with K_ww = G^T diag(w A) G, K_wF = G^T diag(w A), K_FF = sum_p w_p A_p (the
monolithic condensation of Sec. 3.2.3 applied to the full-order system).

Mesh: structured n^d grid on the unit cell (V0 = 1), bilinear Q4 (2D) or
trilinear hex8 (3D) elements with 2^d Gauss points; the material phase of each
element is decided by its centroid (0 = matrix, 1 = inclusion).
"""
import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import law


def _local_corners(d):
    if d == 2:
        return np.array([[0, 0], [1, 0], [1, 1], [0, 1]])
    return np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                     [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]])


def shape_gradients(d, h):
    """Gauss points (2^d, reference coords in [-1,1]^d), d N_a / d X at each
    Gauss point for a cube element of edge h, and the Gauss weight in physical
    volume.  N_a = prod_k (1 + xi_k s_ak)/2 with s_ak = +-1."""
    corners = _local_corners(d)
    s = 2 * corners - 1
    g1 = 1.0 / np.sqrt(3.0)
    gps = np.array(list(itertools.product([-g1, g1], repeat=d)))
    nen = 2 ** d
    dN = np.zeros((len(gps), nen, d))
    for q, xi in enumerate(gps):
        for a in range(nen):
            for k in range(d):
                v = s[a, k] / 2.0
                for m in range(d):
                    if m != k:
                        v *= (1.0 + xi[m] * s[a, m]) / 2.0
                dN[q, a, k] = v * (2.0 / h)
    wgp = (h / 2.0) ** d
    return gps, dN, wgp


def phases_single_inclusion(d, n, vf):
    """Centred circle (2D) / sphere (3D) of volume fraction vf in the unit cell;
    element phase by centroid."""
    r = (vf / np.pi) ** 0.5 if d == 2 else (3.0 * vf / (4.0 * np.pi)) ** (1.0 / 3.0)
    cent = (np.array(list(itertools.product(range(n), repeat=d)))[:, ::-1] + 0.5) / n
    dist = np.linalg.norm(cent - 0.5, axis=1)
    return (dist <= r).astype(np.int64)


def phases_random_inclusions(d, n, centres, radius):
    """Equal circles/spheres at the given centres, periodic images included."""
    cent = (np.array(list(itertools.product(range(n), repeat=d)))[:, ::-1] + 0.5) / n
    ph = np.zeros(len(cent), dtype=np.int64)
    for c in centres:
        dv = cent - c
        dv -= np.round(dv)
        ph[np.linalg.norm(dv, axis=1) <= radius] = 1
    return ph


class PeriodicRVE:
    """Structured periodic RVE.  Element e has lower corner index (ix, iy[, iz])
    with e = ix + n*iy (+ n^2*iz); node v = ix + n*iy (+ n^2*iz) (periodic)."""

    def __init__(self, d, n, phase, moduli):
        self.d, self.n = d, n
        self.g = d * d
        self.V0 = 1.0
        self.phase = np.asarray(phase, dtype=np.int64)
        self.moduli = np.asarray(moduli, dtype=float)   # [n_phase, 2] = (mu, kappa)
        h = 1.0 / n
        _, self.dN, self.wgp = shape_gradients(d, h)     # dN [ngp, nen, d]
        ngp = len(self.dN)
        nen = 2 ** d
        corners = _local_corners(d)
        idx = np.array(list(itertools.product(range(n), repeat=d)))[:, ::-1]  # (ix, iy[, iz])
        ne = len(idx)
        conn = np.zeros((ne, nen), dtype=np.int64)
        stride = n ** np.arange(d)
        for a in range(nen):
            conn[:, a] = (((idx + corners[a]) % n) * stride).sum(axis=1)
        self.conn = conn
        self.n_el = ne
        self.n_ip = ne * ngp
        self.ngp = ngp
        self.ip_weight = np.full(self.n_ip, self.wgp)
        self.ip_phase = np.repeat(self.phase, ngp)
        mu_k = self.moduli[self.ip_phase]
        self.ip_mu, self.ip_kappa = mu_k[:, 0], mu_k[:, 1]
        # DOF numbering: node v, component i -> v*d + i; node 0 fixed
        nn = n ** d
        full = np.arange(nn * d).reshape(nn, d)
        red = np.full(nn * d, -1, dtype=np.int64)
        red[d:] = np.arange(nn * d - d)
        self.n_dof = nn * d - d
        # G: (n_ip*g) x n_dof, row (p, i*d+J) col dof(node, i) = dN[a, J]
        rows, cols, vals = [], [], []
        for e_gp in range(ngp):
            p = np.arange(ne) * ngp + e_gp
            for a in range(nen):
                for i in range(d):
                    dof = red[full[conn[:, a], i]]
                    keep = dof >= 0
                    for J in range(d):
                        rows.append(p[keep] * self.g + i * d + J)
                        cols.append(dof[keep])
                        vals.append(np.full(keep.sum(), self.dN[e_gp, a, J]))
        self.G = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(self.n_ip * self.g, self.n_dof))

    # -- kinematics and quadrature ------------------------------------------
    def F_at_ips(self, Fbar, w):
        d = self.d
        return Fbar.reshape(1, d, d) + (self.G @ w).reshape(self.n_ip, d, d)

    def _block_diag(self, blocks):
        """Block-diagonal sparse matrix of n_ip blocks g x g."""
        g = self.g
        return sp.bsr_matrix((blocks, np.arange(self.n_ip), np.arange(self.n_ip + 1)),
                             shape=(self.n_ip * g, self.n_ip * g)).tocsr()

    def evaluate(self, Fbar, w, need_tangent=True):
        """Residual f (n_dof), Pbar (d x d) and, if asked, K_ww, K_wF, K_FF."""
        d, g = self.d, self.g
        F = self.F_at_ips(Fbar, w)
        P = law.stress(F, self.ip_mu, self.ip_kappa)
        wP = (self.ip_weight[:, None] * P.reshape(self.n_ip, g)).ravel()
        f = self.G.T @ wP
        Pbar = (self.ip_weight[:, None] * P.reshape(self.n_ip, g)).sum(0).reshape(d, d) / self.V0
        if not need_tangent:
            return f, Pbar, F, P
        A = law.tangent(F, self.ip_mu, self.ip_kappa).reshape(self.n_ip, g, g)
        wA = self.ip_weight[:, None, None] * A
        D = self._block_diag(wA)
        Kww = (self.G.T @ D @ self.G).tocsc()
        KwF = self.G.T @ wA.reshape(self.n_ip * g, g)
        KFF = wA.sum(0)
        return f, Pbar, F, P, Kww, np.asarray(KwF), KFF

    # -- full-order Newton at fixed Fbar -------------------------------------
    def solve(self, Fbar, w0=None, tol=None, maxit=40):
        """Micro equilibrium at fixed Fbar.  Returns w, Pbar, Cbar (g x g), its."""
        if tol is None:
            tol = 1e-11 * self.moduli[0, 0] * self.V0
        w = np.zeros(self.n_dof) if w0 is None else w0.copy()
        for it in range(maxit):
            f, Pbar, F, P, Kww, KwF, KFF = self.evaluate(Fbar, w)
            if np.max(np.abs(f)) <= tol:
                lu = spla.splu(Kww)
                Cbar = (KFF - KwF.T @ lu.solve(KwF)) / self.V0
                return w, Pbar, Cbar, it
            w = w - spla.spsolve(Kww, f)
        raise RuntimeError("full-order RVE Newton did not converge")

    def linear_responses(self):
        """Fluctuations answering the n_sigma unit symmetric macro strains of
        the linearized RVE at Fbar = I: w_v = -K_ww^-1 K_wF E_v."""
        d = self.d
        f, Pbar, F, P, Kww, KwF, KFF = self.evaluate(np.eye(d), np.zeros(self.n_dof))
        E = voigt_map(d)
        return -spla.splu(Kww).solve(KwF @ E)


def voigt_pairs(d):
    if d == 2:
        return [(0, 0), (1, 1), (0, 1)]
    return [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


def voigt_map(d):
    """E (g x n_sigma): full row-major components of a symmetric tensor from
    its independent (tensor, not engineering) components."""
    pr = voigt_pairs(d)
    E = np.zeros((d * d, len(pr)))
    for v, (i, j) in enumerate(pr):
        E[i * d + j, v] = 1.0
        E[j * d + i, v] = 1.0
    return E


def to_voigt(U):
    d = U.shape[0]
    return np.array([U[i, j] for (i, j) in voigt_pairs(d)])
