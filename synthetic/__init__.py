"""Seeded synthetic input generators shared by the tests, the benchmark and the
CPU oracle's offline scripts.

This module holds no arithmetic of the hyper-ROM method itself: it only draws
random numbers (stretch tensors, rotations, perturbations, RVE-type labels,
inclusion centres) with numpy's PCG64 generator, so that both the CUDA path and
the oracle can be fed identical inputs.  Every draw takes an explicit seed.
"""
import numpy as np

SEED_BASE = 2306_02687


def rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def voigt_dim(d):
    return 3 if d == 2 else 6


def voigt_pairs(d):
    """Index pairs (i, J) of the independent components of a symmetric d x d
    tensor, in the order used for every stretch vector in this project."""
    if d == 2:
        return [(0, 0), (1, 1), (0, 1)]
    return [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


def sym_from_unit_vector(x, d):
    """Symmetric matrix whose Frobenius norm equals ||x||: off-diagonal entries
    get x/sqrt(2) so that both off-diagonal copies together carry x^2."""
    e = np.zeros((d, d))
    for v, (i, j) in enumerate(voigt_pairs(d)):
        if i == j:
            e[i, i] = x[v]
        else:
            e[i, j] = e[j, i] = x[v] / np.sqrt(2.0)
    return e


def random_sym_in_ball(g, d, radius):
    """Symmetric d x d matrix drawn uniformly (in its n_sigma-dim space with
    the Frobenius metric) from the ball of the given radius."""
    n = voigt_dim(d)
    x = g.standard_normal(n)
    x /= np.linalg.norm(x)
    x *= radius * g.random() ** (1.0 / n)
    return sym_from_unit_vector(x, d)


def random_sym_norm_uniform(g, d, eps_max):
    """Symmetric matrix with random direction and Frobenius norm uniform in
    [0, eps_max] (the batch-stretch recipe of the benchmark workloads)."""
    n = voigt_dim(d)
    x = g.standard_normal(n)
    x /= np.linalg.norm(x)
    x *= eps_max * g.random()
    return sym_from_unit_vector(x, d)


def random_rotation(g, d, max_angle):
    """Rotation by an angle uniform in [-max_angle, max_angle]; in 3D about a
    uniformly random axis (Rodrigues' formula)."""
    th = (2.0 * g.random() - 1.0) * max_angle
    if d == 2:
        c, s = np.cos(th), np.sin(th)
        return np.array([[c, -s], [s, c]])
    ax = g.standard_normal(3)
    ax /= np.linalg.norm(ax)
    k = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    return np.eye(3) + np.sin(th) * k + (1.0 - np.cos(th)) * (k @ k)


def training_paths(seed, d, n_paths, n_steps, eps_max):
    """Monotonic stretch paths U_k = I + (k/n_steps) eps, k = 1..n_steps, with
    eps symmetric and uniform in the Frobenius ball of radius eps_max.
    Returns an array [n_paths, n_steps, d, d]."""
    g = rng(seed)
    out = np.zeros((n_paths, n_steps, d, d))
    for p in range(n_paths):
        e = random_sym_in_ball(g, d, eps_max)
        for k in range(n_steps):
            out[p, k] = np.eye(d) + (k + 1) / n_steps * e
    return out


def fbar_batch(seed, d, n, eps_max, max_angle):
    """Batch of macro deformation gradients F = R (I + eps): stretch with
    ||eps||_F uniform in [0, eps_max], rotation up to max_angle.
    Returns [n, d, d] float64."""
    g = rng(seed)
    out = np.zeros((n, d, d))
    for a in range(n):
        u = np.eye(d) + random_sym_norm_uniform(g, d, eps_max)
        out[a] = random_rotation(g, d, max_angle) @ u
    return out


def inclusion_centres(seed, d, n_incl, radius, gap):
    """Centres of n_incl equal spheres/circles in the periodic unit cell, drawn
    by rejection so that periodic centre distances are >= 2 radius + gap."""
    g = rng(seed)
    centres = []
    tries = 0
    while len(centres) < n_incl:
        tries += 1
        if tries > 200000:
            raise RuntimeError("could not place inclusions")
        c = g.random(d)
        ok = True
        for c2 in centres:
            dv = c - c2
            dv -= np.round(dv)
            if np.linalg.norm(dv) < 2.0 * radius + gap:
                ok = False
                break
        if ok:
            centres.append(c)
    return np.array(centres)


def type_labels(seed, n, n_types):
    return rng(seed).integers(0, n_types, size=n).astype(np.int32)


def perturbation(seed, shape, scale):
    return scale * rng(seed).standard_normal(shape)
