"""Clustered training (Sec. 3.4, Box 2): a simple surrogate material model,
the macro simulation with it, the macro integration points' deformation
paths, and k-means clustering of those paths into the training set.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

  step 1  surrogate: linear elasticity with the initial RVE stiffness, here
          the condensed tangent of the hyper-ROM at Fbar = I (Box 2 names
          "linear elastic, with initial RVE stiffness")
  step 2  the macro problem with the surrogate, Pbar = C0 : (Fbar - I): per
          load step the linear system K du = -R on the free DOFs; the path of
          every macro point is its displacement gradient H = Fbar - I at each
          load step (the set T of the paper holds H(t) trajectories),
          concatenated over the steps
  step 3  k-means (Lloyd): assign every path to the nearest centre (squared
          Euclidean distance, summed over the coordinates in order; ties to
          the lowest index), move every centre to the mean of its paths
          (an empty cluster keeps its centre), until no assignment changes
  step 4  the centres are the training trajectories (reshaped to n_steps
          displacement gradients; their stretches drive the training runs)
Readings: the paper leaves the clustered quantity and the distance open;
the displacement-gradient paths with the Euclidean distance are used, and
the initial centres are given (seeded draws of distinct paths).
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import reduced


def initial_stiffness(rom):
    """C0 = dPbar/dFbar of the hyper-ROM at Fbar = I (g x g)."""
    st = reduced.zero_state(rom)
    st['Uprev'] = np.array([1.0] * rom.d + [0.0] * (rom.ns - rom.d))
    o = reduced.eval_point(rom, np.eye(rom.d), **st)
    return o['dPdF']


def surrogate_paths(problem, C0, n_steps):
    """Paths [n_ip, n_steps * g] of H = Fbar - I under the linear surrogate,
    load factor k / n_steps at step k, and the final displacement."""
    mesh = problem.mesh
    d = mesh.d
    g = d * d
    u = np.zeros((mesh.n_nodes, d))
    paths = np.zeros((mesh.n_ip, n_steps, g))
    Cs = np.repeat(np.asarray(C0)[None], mesh.n_ip, axis=0)
    for k in range(1, n_steps + 1):
        uf = u.reshape(-1)
        uf[problem.presc_dofs] = k / n_steps * problem.presc_vals
        H = (mesh.gradient(u) - np.eye(d)[None]).reshape(mesh.n_ip, g)
        P = np.einsum('pce,pe->pc', Cs, H).reshape(mesh.n_ip, d, d)
        R, K = mesh.assemble(P, Cs)
        Kff = K[problem.free][:, problem.free].tocsc()
        uf[problem.free] += spla.spsolve(Kff, -R[problem.free])
        paths[:, k - 1] = (mesh.gradient(u) - np.eye(d)[None]).reshape(mesh.n_ip, g)
    return paths.reshape(mesh.n_ip, n_steps * g), u


def assign(X, C):
    """Nearest centre of every row of X; distances summed over the
    coordinates in order (the same rounding as a sequential loop)."""
    dist = np.zeros((X.shape[0], C.shape[0]))
    for j in range(X.shape[1]):
        diff = X[:, j][:, None] - C[None, :, j]
        dist = dist + diff * diff
    return np.argmin(dist, axis=1).astype(np.int32), dist


def kmeans(X, C_init, max_iter=100):
    """Lloyd's algorithm from the given centres.  Returns (centres, labels,
    iterations, inertia per iteration)."""
    C = np.array(C_init, dtype=float)
    labels = None
    hist = []
    it = 0
    for it in range(1, max_iter + 1):
        new, dist = assign(X, C)
        hist.append(dist[np.arange(len(X)), new].sum())
        if labels is not None and np.array_equal(new, labels):
            it -= 1
            break
        labels = new
        for c in range(C.shape[0]):
            sel = labels == c
            if sel.any():
                C[c] = X[sel].mean(axis=0)
    else:                                   # out of iterations: labels of the final centres
        labels = assign(X, C)[0]
    _, dist = assign(X, C)
    inertia = dist[np.arange(len(X)), labels].sum()
    return C, labels, it, inertia, hist
