"""The offline (training) stage of the hyper-ROM on the device, planar RVEs
(Sec. 3.2.1 snapshots and POD, Sec. 3.3 empirical cubature): argument
marshalling over the library's offline entry points (include/rverom.h)."""
import ctypes

import numpy as np
import torch

from . import _native
from .api import _ptr, _stream


def rve_snapshots(n, phase, moduli, paths=None, linear=False, tol=None, cg_tol=1e-12, max_newton=40,
                  max_cg=20000, stream=None):
    """Full-order periodic RVE fluctuations along the training paths (device
    [n_paths, n_steps, 2, 2] stretches), or the three linearized responses
    (linear=True).  Returns (X [n_snap, n_dof], info [n_problems, 4])."""
    phase = torch.as_tensor(np.ascontiguousarray(phase, dtype=np.int32), device='cuda')
    mod = np.ascontiguousarray(moduli, dtype=np.float64).reshape(4)
    if tol is None:
        tol = 1e-11 * float(mod[0])
    n_dof = 2 * n * n - 2
    if linear:
        n_paths, n_steps = 3, 1
        pp = None
    else:
        n_paths, n_steps = paths.shape[0], paths.shape[1]
        pp = _ptr(paths.reshape(n_paths, n_steps, 4).contiguous(), torch.float64, (n_paths, n_steps, 4), 'paths')
    X = torch.empty(n_paths * n_steps, n_dof, dtype=torch.float64, device='cuda')
    info = torch.empty(n_paths, 4, dtype=torch.float64, device='cuda')
    _native.check(_native.lib().rve_snapshots(
        n, _ptr(phase, torch.int32, (n * n,), 'phase'), mod.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        n_paths, n_steps, pp, 1 if linear else 0, float(tol), float(cg_tol), int(max_newton), int(max_cg),
        _ptr(X, torch.float64, None, 'X'), _ptr(info, torch.float64, None, 'info'), _stream(stream)),
        'rve_snapshots')
    return X, info
