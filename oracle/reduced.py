"""Hyper-reduced RVE evaluation at one macro integration point, in float64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Follows, step by step:
  a1  polar split Fbar = R U (Sec. 3.2.2, Eq. polar_decomp); the monolithic
      micro update of Sec. 3.2.3, dq = -k~^-1 (r~ + dr~/dU dU), applied with
      the stored s = k~^-1 r~, S = k~^-1 dr~/dU of the previous evaluation:
      q <- q - s - S (U - U_prev)
  a2  F_i = U + B_i q at every ECM point (ROM ansatz Eq. ROM_assumption;
      B_i = grad Phi at ECM point i; hyper-element evaluation of Sec. 4)
  a3  P_i, A_i from the micro law
  a4  r = sum_i w_i B_i^T P_i (Eq. ROMintforce with ECM weights),
      Pbar_U = (1/V0) sum_i w_i P_i (Eq. 2 with the cubature of Sec. 3.3)
  a5  K = sum_i w_i B_i^T A_i B_i (Eq. ROMstiffness), the coupling
      K_qF = sum_i w_i B_i^T A_i = dr/dU and K_FF = sum_i w_i A_i
  a6  static condensation (Sec. 3.2.3): s = K^-1 r, S = K^-1 K_qF E,
      algorithmic stress Pbar_alg = Pbar_U - (1/V0) K_qF^T s and condensed
      tangent C_U = (1/V0)(K_FF - K_qF^T K^-1 K_qF)  (Eq. Biot_Tangent written
      for the first Piola-Kirchhoff stress at U); factorization, no inverse
  a7  Pbar = R Pbar_alg and dPbar/dFbar = dR Pbar_alg + R C_U[dU] through the
      polar derivative.
Reading used for finite rotations: the RVE sees only U and Pbar = R Pbar(U)
(exact objectivity); the Biot/Cauchy conversions are a macro-code interface
detail and are not needed by a total-Lagrangian macro code.
"""
import numpy as np

from . import law, polar as pol, rve as rvemod

OK, DETF_NONPOS, NONSPD_K, NONFINITE, NOT_CONVERGED = 0, 1, 2, 3, 4


class Rom:
    """Hyper-ROM tables of one RVE type: B [m, g, n], w [m], phase [m],
    moduli [n_phase, 2] = (mu, kappa), V0."""

    def __init__(self, B, w, phase, moduli, V0=1.0):
        self.B = np.asarray(B, dtype=float)
        self.w = np.asarray(w, dtype=float)
        self.phase = np.asarray(phase, dtype=np.int64)
        self.moduli = np.asarray(moduli, dtype=float)
        self.V0 = float(V0)
        self.m, self.g, self.n = self.B.shape
        self.d = int(round(np.sqrt(self.g)))
        self.ns = 3 if self.d == 2 else 6

    @staticmethod
    def load(path):
        z = np.load(path)
        return Rom(z['B'], z['w'], z['phase'], z['moduli'], float(z['V0']))

    def with_moduli(self, moduli):
        return Rom(self.B, self.w, self.phase, moduli, self.V0)


def zero_state(rom):
    return dict(q=np.zeros(rom.n), s=np.zeros(rom.n), S=np.zeros((rom.n, rom.ns)),
                Uprev=np.zeros(rom.ns))


def reduced_system(rom, U, q, pointwise=None):
    """a2-a5: returns r, V0*Pbar_U (g), K, K_qF, K_FF, F_i, status.
    pointwise(F [m, d, d]) -> (P [m, d, d], A [m, g, g]) replaces the
    Neo-Hooke law (a history-dependent law at the ECM points)."""
    d, g, m = rom.d, rom.g, rom.m
    F = U.reshape(1, g) + np.einsum('icj,j->ic', rom.B, q)
    F = F.reshape(m, d, d)
    if np.any(np.linalg.det(F) <= 0.0):
        return None, None, None, None, None, F, DETF_NONPOS
    if pointwise is None:
        mu = rom.moduli[rom.phase, 0]
        ka = rom.moduli[rom.phase, 1]
        P = law.stress(F, mu, ka).reshape(m, g)
        A = law.tangent(F, mu, ka).reshape(m, g, g)
    else:
        P, A = pointwise(F)
        P = P.reshape(m, g)
        A = A.reshape(m, g, g)
    wP = rom.w[:, None] * P
    r = np.einsum('icj,ic->j', rom.B, wP)
    VPU = wP.sum(0)
    wA = rom.w[:, None, None] * A
    Y = np.einsum('icd,idk->ick', wA, rom.B)           # w_i A_i B_i
    K = np.einsum('icj,ick->jk', rom.B, Y)
    KqF = np.einsum('icj,icd->jd', rom.B, wA)
    KFF = wA.sum(0)
    if not (np.all(np.isfinite(r)) and np.all(np.isfinite(K))):
        return None, None, None, None, None, F, NONFINITE
    return r, VPU, K, KqF, KFF, F, OK


def eval_point(rom, Fbar, q, s, S, Uprev, pointwise=None):
    """One monolithic evaluation (steps a1-a7).  Returns a dict with Pbar
    (d x d), dPdF (g x g, [out, in] in row-major component order), the new
    state q, s, S, Uprev, rnorm = max|r| and status."""
    d, g = rom.d, rom.g
    V0 = rom.V0
    R, U = pol.polar(Fbar)
    Uv = rvemod.to_voigt(U)
    q = q - s - S @ (Uv - Uprev)
    r, VPU, K, KqF, KFF, F, st = reduced_system(rom, U, q, pointwise)
    out = dict(q=q, status=st)
    if st != OK:
        return out
    try:
        L = np.linalg.cholesky(K)
    except np.linalg.LinAlgError:
        out['status'] = NONSPD_K
        return out
    E = rvemod.voigt_map(d)

    def solve(b):
        return np.linalg.solve(L.T, np.linalg.solve(L, b))

    s_new = solve(r)
    X = solve(KqF)                       # K^-1 K_qF  (n x g)
    S_new = X @ E
    Palg = ((VPU - KqF.T @ s_new) / V0).reshape(d, d)
    CU = (KFF - KqF.T @ X) / V0
    Pbar = R @ Palg
    dPdF = np.zeros((g, g))
    for c in range(g):
        dF = np.zeros(g)
        dF[c] = 1.0
        dR, dU = pol.polar_derivative(R, U, dF.reshape(d, d))
        dP = dR @ Palg + R @ (CU @ dU.ravel()).reshape(d, d)
        dPdF[:, c] = dP.ravel()
    out.update(Pbar=Pbar, dPdF=dPdF, s=s_new, S=S_new, Uprev=Uv,
               rnorm=np.max(np.abs(r)), r=r, Palg=Palg, CU=CU, K=K, KqF=KqF, KFF=KFF,
               R=R, U=U)
    return out


def converge_point(rom, Fbar, q0=None, tol=None, maxit=50):
    """Staggered micro solve at fixed Fbar: repeat the evaluation (which then
    reduces to micro Newton steps q <- q - K^-1 r) until max|r| <= tol.
    Returns the last evaluation dict and the iteration count."""
    if tol is None:
        tol = 1e-12 * rom.moduli[0, 0] * rom.V0
    st = zero_state(rom)
    if q0 is not None:
        st['q'] = np.array(q0, dtype=float)
    R, U = pol.polar(Fbar)
    st['Uprev'] = rvemod.to_voigt(U)
    for it in range(maxit):
        o = eval_point(rom, Fbar, st['q'], st['s'], st['S'], st['Uprev'])
        if o['status'] != OK:
            return o, it
        if o['rnorm'] <= tol:
            return o, it
        st = dict(q=o['q'], s=o['s'], S=o['S'], Uprev=o['Uprev'])
    o['status'] = NOT_CONVERGED
    return o, maxit


def eval_batch(roms, types, Fbar, q, s, S, Uprev):
    """Loop of eval_point over a batch (types[a] selects roms[types[a]]).
    Per-point state arrays are lists of 1-D/2-D arrays (sizes differ per
    type).  Returns a list of result dicts."""
    return [eval_point(roms[types[a]], Fbar[a], q[a], s[a], S[a], Uprev[a])
            for a in range(len(types))]
