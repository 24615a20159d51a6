"""Macro mesh geometry of the synthetic workloads (node coordinates and
element connectivity only; no finite-element arithmetic).

Node order inside an element follows the isoparametric convention used by
both the CUDA macro kernels and the oracle: Q4 counter-clockwise
(-1,-1), (1,-1), (1,1), (-1,1); hex8 the bottom face then the top face.
"""
import numpy as np


def rect(nx, ny, Lx=1.0, Ly=1.0):
    xs, ys = np.linspace(0, Lx, nx + 1), np.linspace(0, Ly, ny + 1)
    X = np.array([[x, y] for y in ys for x in xs])
    conn = []
    for j in range(ny):
        for i in range(nx):
            n0 = j * (nx + 1) + i
            conn.append([n0, n0 + 1, n0 + nx + 2, n0 + nx + 1])
    return X, np.array(conn, dtype=np.int64)


def box(nx, ny, nz, Lx, Ly, Lz):
    xs, ys, zs = np.linspace(0, Lx, nx + 1), np.linspace(0, Ly, ny + 1), np.linspace(0, Lz, nz + 1)
    X = np.array([[x, y, z] for z in zs for y in ys for x in xs])
    conn = []
    sx, sy = nx + 1, (nx + 1) * (ny + 1)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                n0 = k * sy + j * sx + i
                b = [n0, n0 + 1, n0 + sx + 1, n0 + sx]
                conn.append(b + [v + sy for v in b])
    return X, np.array(conn, dtype=np.int64)


def plate_with_hole(nr, nt, half=1.0, radius=0.2):
    """O-grid around a central hole: 4 blocks (one per side of the square
    [-half, half]^2) of nr radial x nt tangential Q4 elements; the blocks share
    their diagonal node lines.  4 nr nt elements."""
    ntot = 4 * nt
    X = np.zeros(((nr + 1) * ntot, 2))
    ids = np.zeros((nr + 1, ntot), dtype=np.int64)
    k = 0
    for t in range(ntot):
        ang = -np.pi / 4 + 2 * np.pi * t / ntot
        c, s = np.cos(ang), np.sin(ang)
        inner = radius * np.array([c, s])
        outer = np.array([c, s]) * half / max(abs(c), abs(s))
        for i in range(nr + 1):
            f = i / nr
            X[k] = (1 - f) * inner + f * outer
            ids[i, t] = k
            k += 1
    conn = []
    for t in range(ntot):
        t1 = (t + 1) % ntot
        for i in range(nr):
            conn.append([ids[i, t], ids[i + 1, t], ids[i + 1, t1], ids[i, t1]])
    return X, np.array(conn, dtype=np.int64)


def boundary_dofs(kind, X):
    """Prescribed DOFs (node * d + i) of the synthetic macro problems, by
    geometry only:
      rect   left edge u_x, bottom edge u_y, right edge u_x (uniaxial tension)
      plate  the normal displacement of the outer square's edges (biaxial)
      box    every DOF of the face x = 0 (clamped) and u_z of the face x = L
             (tip shear of a cantilever)
    Returns (dofs, react_dofs) as int64 arrays: react_dofs are the DOFs whose
    internal forces sum to the reaction of the loaded boundary."""
    d = X.shape[1]
    lo, hi = X.min(0), X.max(0)
    on = lambda k, v: np.nonzero(np.isclose(X[:, k], v))[0]
    if kind == 'rect':
        left, bottom, right = on(0, lo[0]), on(1, lo[1]), on(0, hi[0])
        dofs = np.concatenate([left * d, bottom * d + 1, right * d])
        react = right * d
    elif kind == 'plate':
        xs = np.concatenate([on(0, lo[0]), on(0, hi[0])])
        ys = np.concatenate([on(1, lo[1]), on(1, hi[1])])
        dofs = np.concatenate([xs * d, ys * d + 1])
        react = on(0, hi[0]) * d
    else:
        clamp, tip = on(0, lo[0]), on(0, hi[0])
        dofs = np.concatenate([clamp * d + i for i in range(d)] + [tip * d + 2])
        react = tip * d + 2
    return np.unique(dofs).astype(np.int64), np.unique(react).astype(np.int64)
