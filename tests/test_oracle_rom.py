"""Pins of the ROM machinery (POD with el/inel split, ECM Box 1) and of the
reduced evaluation against the independent full-order FE oracle."""
import numpy as np
import pytest

import synthetic as syn
from oracle import law, rve, rom, reduced, polar

MU, KA = law.mu_kappa_from_E_nu(1.0, 0.3)
MOD = [[MU, KA], [10 * MU, 10 * KA]]


def model(d, n, vf=0.2):
    return rve.PeriodicRVE(d, n, rve.phases_single_inclusion(d, n, vf), MOD)


@pytest.mark.parametrize('d,n', [(2, 4), (3, 2)])
def test_complete_basis_full_integration_equals_full_order(d, n):
    # Phi = I with all Gauss points: the reduced evaluation must be the
    # full-order FE problem (two independent implementations)
    m = model(d, n)
    full = rom.full_integration_rom(m, np.eye(m.n_dof))
    import synthetic
    Fb = synthetic.fbar_batch(5, d, 1, 0.15, 0.4)[0]
    o, _ = reduced.converge_point(full, Fb, tol=1e-13)
    R, U = polar.polar(Fb)
    w, PU, CU, _ = m.solve(U, tol=1e-13)
    assert np.abs(o['Palg'] - PU).max() < 1e-12
    assert np.abs(o['CU'] - CU).max() < 1e-11
    assert np.abs(o['Pbar'] - R @ PU).max() < 1e-12
    _, Pf, _, _ = m.solve(Fb, tol=1e-13)
    assert np.abs(o['Pbar'] - Pf).max() < 1e-12


def test_elastic_modes_give_exact_small_strain_tangent():
    # el/inel split: Phi_el alone recovers the elastic range exactly
    m = model(2, 8)
    Phi_el = np.linalg.svd(m.linear_responses(), full_matrices=False)[0]
    r = rom.full_integration_rom(m, Phi_el)
    o, _ = reduced.converge_point(r, np.eye(2))
    _, _, C, _ = m.solve(np.eye(2))
    E = rve.voigt_map(2)
    assert np.abs(o['CU'] @ E - C @ E).max() < 1e-12


def _paths(d, n_paths, n_steps, eps, seed=3):
    return syn.training_paths(seed, d, n_paths, n_steps, eps)


def test_rom_error_falls_with_modes():
    m = model(2, 12)
    paths = _paths(2, 8, 4, 0.12)
    X = rom.snapshots(m, paths)
    Fb = syn.fbar_batch(99, 2, 1, 0.1, 0.0)[0]
    _, Pf, _, _ = m.solve(Fb)
    errs = []
    for nm in (3, 6, 12):
        r = rom.full_integration_rom(m, rom.pod_basis(m, X, nm))
        o, _ = reduced.converge_point(r, Fb)
        errs.append(np.abs(o['Pbar'] - Pf).max())
    assert errs[0] > errs[1] > errs[2]
    Phi = rom.pod_basis(m, X, 12)
    # orthonormal to rounding (Phi_inel is orthogonal to Phi_el up to the
    # rounding of the projection removed from the snapshots)
    assert np.abs(Phi.T @ Phi - np.eye(12)).max() < 1e-10


def test_pod_split_spans_the_elastic_range_and_the_remaining_snapshots():
    # Eqs. SVD_displacement / snapshots_displacement: Phi_el spans the linear
    # responses to the unit macro strains; Phi_inel is orthogonal to it and
    # is the best rank-k basis of the snapshots with their Phi_el part
    # removed: the projection error equals the sum of the discarded
    # eigenvalues of the Gram matrix of those snapshots (computed here by a
    # symmetric eigen-solver, not an SVD)
    m = model(2, 10)
    X = rom.snapshots(m, _paths(2, 6, 4, 0.12, seed=8))
    Wel = m.linear_responses()
    nel = 3
    for k in (2, 5):
        Phi = rom.pod_basis(m, X, nel + k)
        Pel, Pin = Phi[:, :nel], Phi[:, nel:]
        assert np.linalg.norm(Wel - Pel @ (Pel.T @ Wel)) < 1e-12 * np.linalg.norm(Wel)
        assert np.abs(Pel.T @ Pin).max() < 1e-10
        Xm = X - Wel @ np.linalg.solve(Wel.T @ Wel, Wel.T @ X)       # remove the elastic part
        ev = np.sort(np.linalg.eigvalsh(Xm.T @ Xm))[::-1]
        err2 = np.linalg.norm(Xm - Pin @ (Pin.T @ Xm)) ** 2
        assert abs(err2 - ev[k:].sum()) <= 1e-8 * ev.sum()
    # a basis that skipped the removal of the elastic part would not be
    # orthogonal to it
    Uraw = np.linalg.svd(X, full_matrices=False)[0][:, :2]
    assert np.abs(Pel.T @ Uraw).max() > 1e-3


@pytest.fixture(scope='module')
def small_ecm():
    m = model(2, 8)
    paths = _paths(2, 6, 3, 0.12)
    X = rom.snapshots(m, paths)
    Phi = rom.pod_basis(m, X, 6)
    fk = rom.ecm_training(m, Phi, paths)
    xf = rom.training_matrix(fk, m.ip_weight, m.V0, 6)
    return m, Phi, paths, fk, xf


def test_ecm_invariants(small_ecm):
    m, Phi, paths, fk, xf = small_ecm
    # the full Gauss rule is a feasible point of the ECM system
    assert np.abs(xf @ m.ip_weight).max() < 1e-14
    z, w = rom.ecm(xf, m.V0, 40)
    assert len(z) == 40 and len(set(z.tolist())) == 40
    assert np.all(w > 0)
    assert abs(w.sum() - m.V0) < 1e-12


def test_ecm_exact_beyond_rank():
    # when m~ - 1 exceeds the rank of x_f the selected rule integrates every
    # training integrand exactly (lambda^T w = 0 on the whole row space)
    m = model(2, 4)
    paths = _paths(2, 2, 2, 0.1)
    X = rom.snapshots(m, paths)
    Phi = rom.pod_basis(m, X, 3)
    fk = rom.ecm_training(m, Phi, paths)
    xf = rom.training_matrix(fk, m.ip_weight, m.V0, 3)
    rank = np.linalg.matrix_rank(xf)
    mt = rank + 1
    z, w = rom.ecm(xf, m.V0, mt)
    if len(z) == mt:
        assert np.abs(xf[:, z] @ w).max() < 1e-10
        for f in fk:
            assert np.abs(w @ f[z] - m.ip_weight @ f).max() < 1e-10


def _brute_force_nnls(A, b):
    """min ||A w - b|| over w >= 0 by enumerating the supports: on each
    support the unconstrained least-squares solution (normal equations),
    kept if non-negative; the best feasible one wins."""
    import itertools
    n = A.shape[1]
    best, best_w = np.inf, np.zeros(n)
    for k in range(n + 1):
        for sup in itertools.combinations(range(n), k):
            w = np.zeros(n)
            if k:
                As = A[:, sup]
                ws = np.linalg.solve(As.T @ As, As.T @ b)
                if np.any(ws < -1e-13):
                    continue
                w[list(sup)] = ws
            res = np.linalg.norm(A @ w - b)
            if res < best - 1e-14:
                best, best_w = res, w
    return best_w


def test_ecm_greedy_box1_on_tiny_system(monkeypatch):
    # Box 1 on small random systems J = [lambda 1]^T, b = [0 V0]^T:
    #  - the first pick is the column most aligned with b (brute force);
    #  - one point: the least-squares weight is the projection of b on j_k;
    #  - every non-negative solve of the loop (the NNLS of step 5) equals a
    #    brute-force enumeration of supports, and zero weights are dropped;
    #  - the result has positive weights that are the least-squares solution
    #    on their support (J_z^T (b - J_z w) = 0);
    #  - when the target count is reached with m~ = rows, J_z w = b exactly.
    import scipy.optimize as spo
    calls = []
    real_nnls = spo.nnls

    def nnls(A, b):
        w = real_nnls(A, b)[0]
        calls.append((A.copy(), b.copy(), w.copy()))
        return w, np.linalg.norm(A @ w - b)
    monkeypatch.setattr(rom.spo, 'nnls', nnls)
    reached = 0
    for seed in range(60):
        rng = np.random.default_rng(seed)
        m, k = 9, 2
        lam = np.linalg.qr(rng.standard_normal((m, k)))[0]
        J = np.vstack([lam.T, np.ones((1, m))])
        b = np.zeros(k + 1)
        b[-1] = 1.0
        if seed == 0:
            score0 = (J.T @ b) / np.linalg.norm(J, axis=0)
            z1, w1 = rom.ecm_greedy(J, b, 1)
            assert z1[0] == int(np.argmax(score0))
            jk = J[:, z1[0]]
            assert abs(w1[0] - (jk @ b) / (jk @ jk)) < 1e-14
        z, w = rom.ecm_greedy(J, b, k + 1)
        assert np.all(w > 0) and len(set(z.tolist())) == len(z)
        r = b - J[:, z] @ w
        assert np.abs(J[:, z].T @ r).max() < 1e-12
        if len(z) == k + 1:
            reached += 1
            assert np.abs(r).max() < 1e-13
    assert reached > 10                    # the exact-solve branch is exercised
    assert len(calls) > 5                  # so is the non-negative solve
    for A, bb, w in calls:
        assert np.abs(w - _brute_force_nnls(A, bb)).max() < 1e-10


def test_hyper_rom_converges_to_full_integration(small_ecm):
    m, Phi, paths, fk, xf = small_ecm
    full = rom.full_integration_rom(m, Phi)
    Fb = syn.fbar_batch(17, 2, 1, 0.1, 0.2)[0]
    of, _ = reduced.converge_point(full, Fb)
    errs = []
    for mt in (8, 60):
        z, w = rom.ecm(xf, m.V0, mt)
        o, _ = reduced.converge_point(rom.hyper_rom(m, Phi, z, w), Fb)
        errs.append(np.abs(o['Pbar'] - of['Pbar']).max())
    assert errs[1] < errs[0]
    assert errs[1] < 1e-3 * np.abs(of['Pbar']).max()
