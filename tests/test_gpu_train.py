"""GPU parity of the Biot/Cauchy outputs (Sec. 3.2.2, Appendix A) and of
the clustered training of Box 2 (linear-elastic surrogate macro run, k-means
of the paths) against the float64 oracle, on oracle inputs."""
import numpy as np
import pytest
import torch

import synthetic as syn
from synthetic import meshes
from conftest import rom_path
from oracle import cluster, law, macro, output, reduced

pytestmark = pytest.mark.gpu
rv = pytest.importorskip('paper_2306_02687_gb300')
from paper_2306_02687_gb300 import training  # noqa: E402


def T(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device='cuda')


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize('d', [2, 3])
def test_biot_cauchy_against_oracle_law_inputs(d):
    n = 64
    F = syn.fbar_batch(syn.SEED_BASE + 250 + d, d, n, 0.25, 0.8)
    mu, ka = law.mu_kappa_from_E_nu(1.0, 0.3)
    P = np.array([law.stress(F[a], mu, ka) for a in range(n)]).reshape(n, d * d)
    A = np.array([law.tangent(F[a], mu, ka).reshape(d * d, d * d) for a in range(n)])
    b, cb, s, cs = rv.rve_rom_biot_cauchy(T(F.reshape(n, -1)), T(P), T(A))
    torch.cuda.synchronize()
    got = [x.cpu().numpy() for x in (b, cb, s, cs)]
    for a in range(n):
        ref = output.outputs(F[a], P[a], A[a])
        for k in range(4):
            assert _rel(got[k][a], ref[k]) <= 1e-12, (a, k)


def test_biot_cauchy_of_the_rom_response():
    # homogenized outputs of the 12-mode ROM at oracle-converged states; the
    # Cauchy stress of the ROM is symmetric by construction of Eq. biotstress
    orom = reduced.Rom.load(rom_path('c1'))
    n = 16
    F = syn.fbar_batch(syn.SEED_BASE + 260, 2, n, 0.1, 0.5)
    P = np.zeros((n, 4))
    A = np.zeros((n, 4, 4))
    for a in range(n):
        o, _ = reduced.converge_point(orom, F[a])
        P[a], A[a] = o['Pbar'].ravel(), o['dPdF']
    b, cb, s, cs = rv.rve_rom_biot_cauchy(T(F.reshape(n, 4)), T(P), T(A))
    torch.cuda.synchronize()
    got = [x.cpu().numpy() for x in (b, cb, s, cs)]
    for a in range(n):
        ref = output.outputs(F[a], P[a], A[a])
        for k in range(4):
            assert _rel(got[k][a], ref[k]) <= 1e-12
    # NULL outputs are skipped; a folded point gets NaN
    Fb = F.reshape(n, 4).copy()
    Fb[3] = [-1.0, 0.0, 0.0, 1.0]
    b2, _, s2, _ = rv.rve_rom_biot_cauchy(T(Fb), T(P), T(A))
    torch.cuda.synchronize()
    assert torch.isnan(b2[3]).all() and torch.isfinite(b2[[0, 1, 2, 4]]).all()


def test_surrogate_run_and_kmeans_against_oracle():
    # Box 2: C0 = the ROM's tangent at Fbar = I; the surrogate macro run on
    # the GPU (linear surrogate, assembly, device solve per load step) against
    # the oracle's; then k-means of the oracle's paths on the GPU against the
    # oracle's k-means
    orom = reduced.Rom.load(rom_path('c1'))
    C0 = cluster.initial_stiffness(orom)
    X, conn = meshes.plate_with_hole(8, 8)
    om = macro.MacroMesh(X, conn)
    # biaxial stretch of the plate: normal displacement of the outer edges
    dofs, _ = meshes.boundary_dofs('plate', X)
    vals = np.array([0.15 * X[k // 2, k % 2] for k in dofs])
    prob = macro.Problem(om, dofs, vals, dofs[:1])
    n_steps = 6
    ref_paths, ref_u = cluster.surrogate_paths(prob, C0, n_steps)
    m = rv.macro_mesh_create(X, conn)
    paths, u, infos = training.surrogate_paths(m, T(C0), dofs, vals, n_steps)
    torch.cuda.synchronize()
    assert np.all(infos.cpu().numpy()[:, 2] == 0)
    assert _rel(paths.cpu().numpy(), ref_paths) <= 1e-9
    assert _rel(u.cpu().numpy(), ref_u) <= 1e-9
    k = 8
    seeds = np.sort(syn.rng(syn.SEED_BASE + 270).choice(len(ref_paths), k, replace=False))
    C_o, lab_o, it_o, in_o, _ = cluster.kmeans(ref_paths, ref_paths[seeds])
    centers, labels, its, inertia = training.cluster_paths(T(ref_paths), k, seeds)
    torch.cuda.synchronize()
    assert np.array_equal(labels.cpu().numpy(), lab_o) and its == it_o
    assert _rel(centers.cpu().numpy(), C_o) <= 1e-12
    assert abs(inertia - in_o) <= 1e-12 * in_o


def test_kmeans_random_paths_against_oracle():
    g = syn.rng(syn.SEED_BASE + 280)
    n, dim, k = 20000, 40, 16
    X = g.standard_normal((n, dim)) + 3.0 * g.standard_normal((1, dim)) * (g.random((n, 1)) < 0.3)
    seeds = np.sort(g.choice(n, k, replace=False))
    C_o, lab_o, it_o, in_o, _ = cluster.kmeans(X, X[seeds], max_iter=60)
    centers = T(X[seeds])
    labels, its, inertia = rv.paths_kmeans(T(X), centers, max_iter=60)
    torch.cuda.synchronize()
    assert its == it_o
    assert np.array_equal(labels.cpu().numpy(), lab_o)
    assert _rel(centers.cpu().numpy(), C_o) <= 1e-12
    assert abs(inertia - in_o) <= 1e-12 * in_o
