"""Clustered training (Sec. 3.4, Box 2) on the device: the macro problem
under the linear-elastic surrogate (step 2) and k-means of its paths
(step 3).  Every step runs in the library's kernels (surrogate_linear_eval,
macro_gradient, macro_assemble, macro_solve, paths_kmeans); this module only
sequences the load steps."""
import torch

from . import api


def surrogate_paths(mesh, C0, presc_dofs, presc_vals, n_steps, tol=1e-13, max_iter=50000):
    """Paths [n_ip, n_steps * g] of H = Fbar - I at every macro point under
    Pbar = C0 (Fbar - I), prescribed DOFs at k / n_steps of presc_vals at
    load step k (one Newton correction per step solves the linear problem).
    Returns (paths, u) as device tensors."""
    dev = C0.device
    d, g = mesh.dim, mesh.g
    u = torch.zeros(mesh.n_nodes, d, dtype=torch.float64, device=dev)
    free = torch.ones(mesh.n_dof, dtype=torch.uint8, device=dev)
    idx = torch.as_tensor(presc_dofs, dtype=torch.int64, device=dev)
    vals = torch.as_tensor(presc_vals, dtype=torch.float64, device=dev)
    free[idx] = 0
    Fbar = torch.empty(mesh.n_ip, g, dtype=torch.float64, device=dev)
    Pbar = torch.empty_like(Fbar)
    dPdF = torch.empty(mesh.n_ip, g, g, dtype=torch.float64, device=dev)
    R = torch.empty(mesh.n_dof, dtype=torch.float64, device=dev)
    Kv = torch.empty(mesh.nnz, dtype=torch.float64, device=dev)
    paths = torch.empty(mesh.n_ip, n_steps, g, dtype=torch.float64, device=dev)
    eye = torch.eye(d, dtype=torch.float64, device=dev).reshape(g)
    infos = []
    for k in range(1, n_steps + 1):
        u.view(-1)[idx] = k / n_steps * vals
        api.macro_gradient(mesh, u, Fbar)
        api.surrogate_linear_eval(C0, Fbar, Pbar, dPdF)
        api.macro_assemble(mesh, Pbar, dPdF, R, Kv)
        _, info = api.macro_solve(mesh, Kv, R, free, u=u, tol=tol, max_iter=max_iter)
        infos.append(info)
        api.macro_gradient(mesh, u, Fbar)
        paths[:, k - 1] = Fbar - eye
    return paths.reshape(mesh.n_ip, n_steps * g), u, torch.stack(infos)


def cluster_paths(paths, k, seed_rows, max_iter=200):
    """k-means of the paths from the rows seed_rows (k distinct indices) as
    initial centres; returns (centres [k][n_steps * g], labels, updates,
    inertia).  The centres are the training trajectories."""
    centers = paths[torch.as_tensor(seed_rows, dtype=torch.int64, device=paths.device)].clone()
    labels, its, inertia = api.paths_kmeans(paths, centers, max_iter=max_iter)
    return centers, labels, its, inertia
