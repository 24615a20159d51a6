"""Pins of the oracle's Biot/Cauchy outputs (Sec. 3.2.2, Eqs. workconjugacy
and biotstress; Appendix A) and of its clustered training (Sec. 3.4, Box 2):
identities and closed forms the paper and the mechanics fix, independent of
the formulas being tested."""
import numpy as np
import pytest

import synthetic as syn
from synthetic import meshes
from conftest import rom_path
from oracle import cluster, law, macro, output, polar, reduced, rve

MU, KA = law.mu_kappa_from_E_nu(1.0, 0.3)
LAM = KA - 2.0 * MU / 3.0


def _law(F):
    d = F.shape[0]
    P = law.stress(F, MU, KA)
    A = law.tangent(F, MU, KA).reshape(d * d, d * d)
    return P, A


def _sym_from_voigt(v, d):
    T = np.zeros((d, d))
    for w, (i, j) in enumerate(syn.voigt_pairs(d)):
        T[i, j] = T[j, i] = v[w]
    return T


@pytest.mark.parametrize('d', [2, 3])
def test_biot_stress_is_work_conjugate_to_the_stretch(d):
    # Eq. workconjugacy: T : dU = P : dF for every dF = R dU (dU symmetric)
    F = syn.fbar_batch(syn.SEED_BASE + 200 + d, d, 1, 0.2, 0.6)[0]
    R, U = polar.polar(F)
    P, A = _law(F)
    T = _sym_from_voigt(output.biot_stress(F, P), d)
    for k in range(4):
        dU = syn.random_sym_in_ball(syn.rng(k), d, 1.0)
        assert abs(np.sum(T * dU) - np.sum(P * (R @ dU))) <= 1e-14 * np.abs(P).max()


@pytest.mark.parametrize('d', [2, 3])
def test_cauchy_from_biot_is_the_true_stress(d):
    # for the pointwise law (P F^T symmetric) the inversion of Eq. biotstress
    # gives sigma = P F^T / J
    F = syn.fbar_batch(syn.SEED_BASE + 210 + d, d, 1, 0.2, 0.6)[0]
    P, A = _law(F)
    T = output.biot_stress(F, P)
    sig = _sym_from_voigt(output.cauchy_stress(F, T), d)
    ref = P @ F.T / np.linalg.det(F)
    assert np.abs(sig - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize('d', [2, 3])
def test_tangents_at_the_reference_state_are_hooke(d):
    # at F = I both tangents are the small-strain isotropic elasticity in
    # tensor components: lam + 2 mu / lam on the normal block, 2 mu on shear
    F = np.eye(d)
    P, A = _law(F)
    CB = output.biot_tangent(F, A)
    CS = output.cauchy_tangent(F, CB)
    ns = 3 if d == 2 else 6
    ref = np.zeros((ns, ns))
    ref[:d, :d] = LAM
    ref[np.arange(d), np.arange(d)] += 2 * MU
    ref[np.arange(d, ns), np.arange(d, ns)] = 2 * MU
    assert np.abs(CB - ref).max() < 1e-14
    assert np.abs(CS - ref).max() < 1e-14


@pytest.mark.parametrize('d', [2, 3])
def test_biot_tangent_is_the_derivative_of_the_biot_stress(d):
    # C^B against central differences of T(U) at fixed R, with the law
    F = syn.fbar_batch(syn.SEED_BASE + 220 + d, d, 1, 0.2, 0.6)[0]
    R, U = polar.polar(F)
    _, A = _law(F)
    CB = output.biot_tangent(F, A)
    h = 1e-6
    for w, (i, j) in enumerate(syn.voigt_pairs(d)):
        E = np.zeros((d, d))
        E[i, j] = E[j, i] = 1.0
        Tp = output.biot_stress(R @ (U + h * E), law.stress(R @ (U + h * E), MU, KA))
        Tm = output.biot_stress(R @ (U - h * E), law.stress(R @ (U - h * E), MU, KA))
        assert np.abs((Tp - Tm) / (2 * h) - CB[:, w]).max() <= 1e-8 * np.abs(CB).max()


@pytest.mark.parametrize('d', [2, 3])
def test_outputs_are_objective(d):
    # a superposed rotation Q leaves T and C^B unchanged and rotates sigma
    F = syn.fbar_batch(syn.SEED_BASE + 230 + d, d, 1, 0.2, 0.3)[0]
    Q = syn.random_rotation(syn.rng(9), d, 0.9)
    P, A = _law(F)
    P2, A2 = _law(Q @ F)
    T1, C1, s1, _ = output.outputs(F, P, A)
    T2, C2, s2, _ = output.outputs(Q @ F, P2, A2)
    assert np.abs(T1 - T2).max() < 1e-13 and np.abs(C1 - C2).max() < 1e-12
    S1 = _sym_from_voigt(s1, d)
    S2 = _sym_from_voigt(s2, d)
    assert np.abs(Q @ S1 @ Q.T - S2).max() < 1e-13


def test_kmeans_recovers_separated_clusters():
    g = syn.rng(syn.SEED_BASE + 240)
    k, dim, per = 5, 12, 80
    means = 10.0 * g.standard_normal((k, dim))
    X = np.vstack([means[c] + 0.1 * g.standard_normal((per, dim)) for c in range(k)])
    truth = np.repeat(np.arange(k), per)
    perm = g.permutation(len(X))
    X, truth = X[perm], truth[perm]
    init = np.array([X[np.nonzero(truth == c)[0][0]] for c in range(k)])
    C, labels, it, inertia, hist = cluster.kmeans(X, init)
    assert np.array_equal(labels, truth)
    for c in range(k):
        assert np.abs(C[c] - means[c]).max() < 0.1 * 4 / np.sqrt(per) * 3
        assert np.allclose(C[c], X[truth == c].sum(0) / per, rtol=0, atol=1e-12)


def test_kmeans_decreases_inertia_and_ends_at_a_fixed_point():
    g = syn.rng(syn.SEED_BASE + 241)
    X = g.standard_normal((300, 7))
    init = X[g.choice(300, 6, replace=False)]
    C, labels, it, inertia, hist = cluster.kmeans(X, init)
    assert all(b <= a + 1e-12 for a, b in zip(hist, hist[1:]))
    for p in range(len(X)):                    # brute force: own centre is the nearest
        dd = [np.linalg.norm(X[p] - C[c]) for c in range(len(C))]
        assert dd[labels[p]] <= min(dd) + 1e-12
    C1, l1, _, _, _ = cluster.kmeans(X, X[:1])
    assert np.allclose(C1[0], X.mean(0), atol=1e-14) and np.all(l1 == 0)


def test_surrogate_paths_are_linear_in_the_load():
    # the linear surrogate: the path at step k is k / n of the final one,
    # and the initial stiffness is major-symmetric and blind to rotations
    orom = reduced.Rom.load(rom_path('c1'))
    C0 = cluster.initial_stiffness(orom)
    assert np.abs(C0 - C0.T).max() <= 1e-12 * np.abs(C0).max()
    W = np.array([0.0, 1.0, -1.0, 0.0])               # skew H
    assert np.abs(C0 @ W).max() <= 1e-12 * np.abs(C0).max()
    X, conn = meshes.rect(5, 4)
    prob = macro.uniaxial_problem(macro.MacroMesh(X, conn), 0.1)
    n = 4
    paths, u = cluster.surrogate_paths(prob, C0, n)
    P = paths.reshape(len(paths), n, 4)
    for k in range(n):
        assert np.abs(P[:, k] - (k + 1) / n * P[:, -1]).max() <= 1e-12 * np.abs(P).max()
