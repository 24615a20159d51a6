"""History-dependent micro law at the ECM points: small-strain J2 (von Mises)
plasticity with linear isotropic hardening, the matrix law of Example 1
(Sec. 5.1: yield stress 0.01 E, hardening modulus 0.016 E, nu = 0.3, elastic
inclusions with 10 E), under plane strain, with the hyper-reduced evaluation
that carries one history record per ECM point.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Law (radial return, backward Euler), strain eps = sym(F - I) embedded in 3D
(plane strain: eps_33 = eps_13 = eps_23 = 0), history (eps_p, alpha):
  trial      s_tr = 2 mu (dev eps - eps_p),  f = |s_tr| - sqrt(2/3) (sy0 + h alpha)
  elastic    f <= 0:  sigma = kappa tr(eps) I + s_tr,  C = kappa I(x)I + 2 mu I_dev
  plastic    dgam = f / (2 mu + 2 h / 3),  n = s_tr / |s_tr|
             s = s_tr - 2 mu dgam n,  eps_p += dgam n,  alpha += sqrt(2/3) dgam
             C = kappa I(x)I + 2 mu b I_dev - 2 mu c n(x)n,
             b = 1 - 2 mu dgam / |s_tr|,  c = 1 / (1 + h / (3 mu)) - (1 - b)
The ROM uses sigma in the place of P and C as dP/dF (small strain, so the
in-plane block of C with its minor symmetry).  History records are
[eps_p 11, 22, 33, 12, 13, 23, alpha]; a phase with sy0 = inf is elastic.
The evaluation is the monolithic step of reduced.eval_point with this law,
every ECM point's return mapping starting from the history of the last
converged load step; the new records are returned and committed by the
driver once the load step has converged.
"""
import numpy as np

from . import reduced, rve as rvemod

NH = 7
_VP = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


def _to_sym(v):
    E = np.zeros((3, 3))
    for k, (i, j) in enumerate(_VP):
        E[i, j] = E[j, i] = v[k]
    return E


def _from_sym(E):
    return np.array([E[i, j] for (i, j) in _VP])


def return_map(eps, hist, mu, kappa, sy0, h):
    """eps (3 x 3 symmetric), hist [7] -> (sigma 3x3, C [3,3,3,3], new hist)."""
    I = np.eye(3)
    ep = _to_sym(hist[:6])
    alpha = hist[6]
    tr = np.trace(eps)
    dev = eps - tr / 3.0 * I
    s_tr = 2.0 * mu * (dev - ep)
    nrm = np.sqrt(np.sum(s_tr * s_tr))
    IxI = np.einsum('ij,kl->ijkl', I, I)
    Isym = 0.5 * (np.einsum('ik,jl->ijkl', I, I) + np.einsum('il,jk->ijkl', I, I))
    Idev = Isym - IxI / 3.0
    f = nrm - np.sqrt(2.0 / 3.0) * (sy0 + h * alpha)
    if not np.isfinite(sy0) or f <= 0.0:
        return kappa * tr * I + s_tr, kappa * IxI + 2.0 * mu * Idev, np.array(hist, dtype=float)
    dg = f / (2.0 * mu + 2.0 * h / 3.0)
    n = s_tr / nrm
    s = s_tr - 2.0 * mu * dg * n
    new = np.zeros(NH)
    new[:6] = _from_sym(ep + dg * n)
    new[6] = alpha + np.sqrt(2.0 / 3.0) * dg
    b = 1.0 - 2.0 * mu * dg / nrm
    c = 1.0 / (1.0 + h / (3.0 * mu)) - (1.0 - b)
    C = kappa * IxI + 2.0 * mu * b * Idev - 2.0 * mu * c * np.einsum('ij,kl->ijkl', n, n)
    return kappa * tr * I + s, C, new


def pointwise(rom, plastic, hist, new_hist):
    """Pointwise law of the ECM points for reduced.reduced_system: plastic
    [n_phase, 2] = (sy0, h) per phase; hist [m, 7] the converged records;
    new_hist (filled) the updated records."""
    d = rom.d

    def law(F):
        m = F.shape[0]
        P = np.zeros((m, d, d))
        A = np.zeros((m, d * d, d * d))
        for i in range(m):
            eps = np.zeros((3, 3))
            H = F[i] - np.eye(d)
            eps[:d, :d] = 0.5 * (H + H.T)
            ph = rom.phase[i]
            mu, ka = rom.moduli[ph]
            sig, C, new_hist[i] = return_map(eps, hist[i], mu, ka, plastic[ph][0], plastic[ph][1])
            P[i] = sig[:d, :d]
            A[i] = C[:d, :d, :d, :d].reshape(d * d, d * d)
        return P, A
    return law


def eval_point(rom, plastic, Fbar, q, s, S, Uprev, hist):
    """One monolithic evaluation with the J2 law; returns the dict of
    reduced.eval_point plus 'hist' (the records after the return mappings)."""
    new_hist = np.array(hist, dtype=float)
    o = reduced.eval_point(rom, Fbar, q, s, S, Uprev, pointwise=pointwise(rom, plastic, hist, new_hist))
    o['hist'] = new_hist
    return o


def driver(problem, rom, plastic, load_factors, tol=1e-10, maxit=30):
    """Monolithic load-stepped Newton with history (one RVE type): the
    prescribed DOFs at load factor lam of their values per step; histories
    committed after every converged step.  Returns the reactions, the
    Newton iteration counts and the final displacement."""
    mesh = problem.mesh
    d, nip = mesh.d, mesh.n_ip
    st = []
    for a in range(nip):
        z = reduced.zero_state(rom)
        z['Uprev'] = rvemod.to_voigt(np.eye(d))
        st.append(z)
    hist = np.zeros((nip, rom.m, NH))
    u = np.zeros((mesh.n_nodes, d))
    reactions, iters = [], []
    import scipy.sparse.linalg as spla
    for lam in load_factors:
        uf = u.reshape(-1)
        uf[problem.presc_dofs] = lam * problem.presc_vals
        for it in range(maxit + 1):
            Fbar = mesh.gradient(u)
            outs = [eval_point(rom, plastic, Fbar[a], hist=hist[a], **st[a]) for a in range(nip)]
            if any(o['status'] != reduced.OK for o in outs):
                raise RuntimeError("micro evaluation failed")
            for a in range(nip):
                st[a] = dict(q=outs[a]['q'], s=outs[a]['s'], S=outs[a]['S'], Uprev=outs[a]['Uprev'])
            R, K = mesh.assemble(np.array([o['Pbar'] for o in outs]), np.array([o['dPdF'] for o in outs]))
            rmax = max(o['rnorm'] for o in outs)
            Rf = R[problem.free]
            if (np.max(np.abs(Rf)) <= tol * max(1.0, np.max(np.abs(R[problem.presc_dofs])))
                    and rmax <= tol * rom.moduli[0, 0] * rom.V0):
                break
            if it == maxit:
                raise RuntimeError("macro Newton did not converge")
            uf = u.reshape(-1)
            uf[problem.free] += spla.spsolve(K[problem.free][:, problem.free].tocsc(), -Rf)
        hist = np.array([o['hist'] for o in outs])
        reactions.append(R[problem.react_dofs].sum())
        iters.append(it)
    return dict(reactions=np.array(reactions), iters=iters, u=u, hist=hist, state=st)

