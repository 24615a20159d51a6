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


def pod_modes(X, W_el, n_modes, stream=None):
    """POD with the elastic/inelastic split (device): returns (Phi
    [n_modes, n_dof], eigenvalues [n_snap], info [2])."""
    n_snap, n_dof = X.shape
    n_el = W_el.shape[0]
    Phi = torch.empty(n_modes, n_dof, dtype=torch.float64, device='cuda')
    eig = torch.empty(n_snap, dtype=torch.float64, device='cuda')
    info = torch.zeros(2, dtype=torch.float64, device='cuda')
    _native.check(_native.lib().pod_modes(
        n_dof, n_snap, _ptr(X.contiguous(), torch.float64, None, 'X'), n_el,
        _ptr(W_el.contiguous(), torch.float64, None, 'W_el'), n_modes, _ptr(Phi, torch.float64, None, 'Phi'),
        _ptr(eig, torch.float64, None, 'eig'), _ptr(info, torch.float64, None, 'info'), _stream(stream)),
        'pod_modes')
    return Phi, eig, info


def mode_gradients(n, Phi, stream=None):
    n_modes = Phi.shape[0]
    B = torch.empty(n * n * 4, 4, n_modes, dtype=torch.float64, device='cuda')
    _native.check(_native.lib().rve_mode_gradients(n, n_modes, _ptr(Phi.contiguous(), torch.float64, None, 'Phi'),
                                                   _ptr(B, torch.float64, None, 'B'), _stream(stream)),
                  'rve_mode_gradients')
    return B


def ecm_training_matrix(n, phase, moduli, B, U, q, stream=None):
    n_modes = B.shape[2]
    n_snap = U.shape[0]
    phase = torch.as_tensor(np.ascontiguousarray(phase, dtype=np.int32), device='cuda')
    mod = np.ascontiguousarray(moduli, dtype=np.float64).reshape(4)
    xf = torch.empty(n_snap * (n_modes + 4), n * n * 4, dtype=torch.float64, device='cuda')
    _native.check(_native.lib().ecm_training_matrix(
        n, _ptr(phase, torch.int32, None, 'phase'), mod.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n_modes,
        _ptr(B.contiguous(), torch.float64, None, 'B'), n_snap, _ptr(U.contiguous(), torch.float64, None, 'U'),
        _ptr(q.contiguous(), torch.float64, None, 'q'), _ptr(xf, torch.float64, None, 'xf'), _stream(stream)),
        'ecm_training_matrix')
    return xf


def ecm_select(xf, V0, m_target, Omega, power_its=2, stream=None):
    """Returns (z [n_sel] int64 host, w [n_sel] host, info [4])."""
    n_rows, m = xf.shape
    k = Omega.shape[1]
    z = torch.empty(m_target, dtype=torch.int32, device='cuda')
    w = torch.empty(m_target, dtype=torch.float64, device='cuda')
    nsel = ctypes.c_int32()
    info = (ctypes.c_double * 4)()
    _native.check(_native.lib().ecm_select(
        m, n_rows, _ptr(xf, torch.float64, None, 'xf'), float(V0), int(m_target),
        _ptr(Omega.contiguous(), torch.float64, None, 'Omega'), k, int(power_its),
        _ptr(z, torch.int32, None, 'z'), _ptr(w, torch.float64, None, 'w'), ctypes.byref(nsel), info,
        _stream(stream)), 'ecm_select')
    ns = nsel.value
    return z[:ns].cpu().numpy().astype(np.int64), w[:ns].cpu().numpy(), list(info)


def converge_full_rom(rom_full, paths, n_iter=12, stream=None):
    """Fully integrated ROM (dict of host tables) along the training paths
    on the device: one macro point per path, each load step from the
    previous amplitudes with fresh s, S (the staggered micro solve of the
    ECM training runs).  Returns (U [n_snap, 4], q [n_snap, n_modes], rnorm max)."""
    from . import api
    n_paths, n_steps = paths.shape[0], paths.shape[1]
    h = api.rve_rom_create(2, [rom_full], 1.0)
    q, s, S, Uv = h.zero_state(n_paths)
    Pbar, dPdF, rnorm, status = h.outputs(n_paths)
    Us, qs = [], []
    worst = 0.0
    for k in range(n_steps):
        F = paths[:, k].reshape(n_paths, 4).contiguous()
        s.zero_()
        S.zero_()
        Uv[:, 0], Uv[:, 1], Uv[:, 2] = F[:, 0], F[:, 3], 0.5 * (F[:, 1] + F[:, 2])
        for _ in range(n_iter):
            api.rve_rom_eval_batch(h, F, q, s, S, Uv, Pbar, dPdF, rnorm, status, precision='fp64', stream=stream)
        if int(status.max().item()) != 0:
            raise RuntimeError('fully integrated ROM failed along a training path')
        worst = max(worst, float(rnorm.max().item()))
        Us.append(F.clone())
        qs.append(q.clone())
    h.destroy()
    U = torch.stack(Us, 1).reshape(n_paths * n_steps, 4)
    qq = torch.stack(qs, 1).reshape(n_paths * n_steps, -1)
    return U, qq, worst


def build_hyper_rom(n, phase, moduli, paths, n_modes, m_target, omega_seed_rows=None, power_its=2, oversample=10,
                    rng=None):
    """The whole offline stage on the device for an n x n planar RVE:
    snapshots along the training paths (host or device [n_paths, n_steps, 2, 2]),
    linearized responses, POD, fully integrated ROM training runs, ECM
    training matrix, empirical cubature.  Returns the hyper-ROM tables (host
    dict B, w, phase, moduli, V0) and a dict of stage outputs and timings."""
    import time
    t = {}
    paths = torch.as_tensor(np.ascontiguousarray(paths, dtype=np.float64), device='cuda')
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X, info_s = rve_snapshots(n, phase, moduli, paths)
    W, info_l = rve_snapshots(n, phase, moduli, linear=True, cg_tol=1e-14)
    torch.cuda.synchronize()
    t['snapshots_s'] = time.perf_counter() - t0
    t0 = time.perf_counter()
    Phi, eig, info_p = pod_modes(X, W, n_modes)
    B = mode_gradients(n, Phi)
    torch.cuda.synchronize()
    t['pod_s'] = time.perf_counter() - t0
    t0 = time.perf_counter()
    nip = n * n * 4
    ph = np.repeat(np.asarray(phase, dtype=np.int32), 4)
    rom_full = dict(B=B.cpu().numpy(), w=np.full(nip, 1.0 / (4 * n * n)), phase=ph,
                    moduli=np.asarray(moduli, dtype=np.float64), V0=1.0)
    U, q, rmax = converge_full_rom(rom_full, paths)
    xf = ecm_training_matrix(n, phase, moduli, B, U, q)
    torch.cuda.synchronize()
    t['ecm_training_s'] = time.perf_counter() - t0
    t0 = time.perf_counter()
    k = m_target - 1 + oversample
    if rng is None:
        rng = np.random.default_rng(0)
    Omega = torch.tensor(rng.standard_normal((xf.shape[0], k)), device='cuda')
    z, w, info_e = ecm_select(xf, 1.0, m_target, Omega, power_its=power_its)
    t['ecm_select_s'] = time.perf_counter() - t0
    order = np.argsort(z)
    z, w = z[order], w[order]
    rom = dict(B=rom_full['B'][z], w=w, phase=ph[z], moduli=rom_full['moduli'], V0=1.0)
    stages = dict(X=X, W=W, Phi=Phi, eig=eig, xf=xf, U=U, q=q, z=z, info_snap=info_s.cpu().numpy(),
                  info_lin=info_l.cpu().numpy(), info_pod=info_p.cpu().numpy(), info_ecm=info_e,
                  rom_rnorm_max=rmax, times=t)
    return rom, stages
