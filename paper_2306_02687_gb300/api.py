"""Thin Python binding of librverom (include/rverom.h).

Argument marshalling only: every step of the hyper-ROM path runs in the CUDA
kernels of the native library.  Tensors are torch CUDA tensors (device memory
and streams come from PyTorch); each function checks dtype, device, shape and
contiguity, passes raw pointers and the current CUDA stream, and raises on a
non-zero return code.
"""
import ctypes

import numpy as np
import torch

from . import _native

FP64 = 0
MIXED = 1
_PREC = {'fp64': FP64, 'mixed': MIXED, FP64: FP64, MIXED: MIXED}


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t, dtype, shape=None, name='tensor'):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError('%s must be a CUDA tensor' % name)
    if t.dtype != dtype:
        raise TypeError('%s must be %s, got %s' % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError('%s must be contiguous' % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError('%s must have shape %s, got %s' % (name, tuple(shape), tuple(t.shape)))
    return ctypes.c_void_p(t.data_ptr())


def load_rom_file(path):
    """Host arrays of a ROM file: dict(B, w, phase, moduli, V0)."""
    z = np.load(path)
    return dict(B=np.ascontiguousarray(z['B'], dtype=np.float64),
                w=np.ascontiguousarray(z['w'], dtype=np.float64),
                phase=np.ascontiguousarray(z['phase'], dtype=np.int32),
                moduli=np.ascontiguousarray(z['moduli'], dtype=np.float64),
                V0=float(z['V0']))


class RomHandle:
    """Owns an rverom_t (device copies of the ROM tables of n_types types)."""

    def __init__(self, ptr, dim, n_types, nmax, V0):
        self.ptr = ptr
        self.dim = dim
        self.g = dim * dim
        self.ns = 3 if dim == 2 else 6
        self.n_types = n_types
        self.nmax = nmax
        self.V0 = V0

    def destroy(self):
        if self.ptr:
            _native.check(_native.lib().rve_rom_destroy(self.ptr), 'rve_rom_destroy')
            self.ptr = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def zero_state(self, n, Fbar=None):
        """Fresh per-point state tensors (q, s, S, Uprev) on the current device;
        Uprev holds the Voigt stretch of I (or of the polar stretch of Fbar
        when given, computed on the host only for initialization)."""
        dev = torch.device('cuda')
        q = torch.zeros(n, self.nmax, dtype=torch.float64, device=dev)
        s = torch.zeros_like(q)
        S = torch.zeros(n, self.nmax, self.ns, dtype=torch.float64, device=dev)
        U = torch.zeros(n, self.ns, dtype=torch.float64, device=dev)
        U[:, :self.dim] = 1.0
        return q, s, S, U

    def outputs(self, n):
        dev = torch.device('cuda')
        return (torch.empty(n, self.g, dtype=torch.float64, device=dev),
                torch.empty(n, self.g, self.g, dtype=torch.float64, device=dev),
                torch.empty(n, dtype=torch.float64, device=dev),
                torch.empty(n, dtype=torch.int32, device=dev))


def rve_rom_create(dim, types, V0=1.0):
    """types: list of dicts with B [m][g][n], w [m], phase [m], moduli [2][2]."""
    n_types = len(types)
    descs = (_native.TypeDesc * n_types)()
    keep = []
    for t, ty in enumerate(types):
        B = np.ascontiguousarray(ty['B'], dtype=np.float64)
        w = np.ascontiguousarray(ty['w'], dtype=np.float64)
        ph = np.ascontiguousarray(ty['phase'], dtype=np.int32)
        mod = np.asarray(ty['moduli'], dtype=np.float64)
        if B.ndim != 3 or B.shape[1] != dim * dim or B.shape[0] != w.shape[0] or ph.shape != w.shape:
            raise ValueError('bad ROM table shapes for type %d' % t)
        keep += [B, w, ph]
        d = descs[t]
        d.n_modes = B.shape[2]
        d.n_ecm = B.shape[0]
        d.B = B.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.w = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.phase = ph.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        for a in range(2):
            for b in range(2):
                d.moduli[a][b] = float(mod[a, b])
    out = ctypes.c_void_p()
    L = _native.lib()
    torch.cuda.current_device()  # make sure the CUDA context exists on the current device
    _native.check(L.rve_rom_create(dim, n_types, descs, float(V0), ctypes.byref(out)), 'rve_rom_create')
    nmax = ctypes.c_int32()
    _native.check(L.rve_rom_nmax(out, ctypes.byref(nmax)), 'rve_rom_nmax')
    return RomHandle(out, dim, n_types, nmax.value, float(V0))


def rve_rom_set_moduli(h, type_id, moduli):
    m = np.ascontiguousarray(moduli, dtype=np.float64).reshape(4)
    _native.check(_native.lib().rve_rom_set_moduli(h.ptr, int(type_id),
                                                   m.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                  'rve_rom_set_moduli')


def rve_rom_autotune(h, precision='mixed', n_sample=16384, stream=None):
    """Time the compiled tile configurations of every RVE type on a synthetic
    sample and keep the fastest; returns the times [n_types][candidates]
    in ms (-1 where a type has fewer candidates, -2 for a candidate rejected
    because a point of the sample did not end with status OK)."""
    ms = np.zeros((h.n_types, 4), dtype=np.float32)
    _native.check(_native.lib().rve_rom_autotune(h.ptr, _PREC[precision], int(n_sample),
                                                 ms.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                 _stream(stream)), 'rve_rom_autotune')
    return ms


def rve_rom_select_kernel(h, type_id, precision, candidate=-1):
    """Pin a tile configuration (candidate >= 0) or just query; returns the
    number of compiled configurations for this type and precision."""
    nc = ctypes.c_int32()
    _native.check(_native.lib().rve_rom_select_kernel(h.ptr, int(type_id), _PREC[precision], int(candidate),
                                                      ctypes.byref(nc)), 'rve_rom_select_kernel')
    return nc.value


def rve_rom_kernel_info(h, type_id, precision, candidate=-1):
    """(name, kernel launches per call) of a forward candidate; candidate < 0
    is the one currently used for this type and precision."""
    buf = ctypes.create_string_buffer(128)
    nl = ctypes.c_int32()
    _native.check(_native.lib().rve_rom_kernel_info(h.ptr, int(type_id), _PREC[precision], int(candidate), buf,
                                                    len(buf), ctypes.byref(nl)), 'rve_rom_kernel_info')
    return buf.value.decode(), nl.value


def rve_rom_eval_batch(h, Fbar, q, s, S, Uprev, Pbar, dPdF, rnorm, status, type=None,
                       precision='mixed', stream=None):
    n = Fbar.shape[0]
    g, ns, nm = h.g, h.ns, h.nmax
    args = [_ptr(type, torch.int32, (n,), 'type') if type is not None else None,
            _ptr(Fbar, torch.float64, (n, g), 'Fbar'),
            _ptr(q, torch.float64, (n, nm), 'q'), _ptr(s, torch.float64, (n, nm), 's'),
            _ptr(S, torch.float64, (n, nm, ns), 'S'), _ptr(Uprev, torch.float64, (n, ns), 'Uprev'),
            _ptr(Pbar, torch.float64, (n, g), 'Pbar'), _ptr(dPdF, torch.float64, (n, g, g), 'dPdF'),
            _ptr(rnorm, torch.float64, (n,), 'rnorm'), _ptr(status, torch.int32, (n,), 'status')]
    rc = _native.lib().rve_rom_eval_batch(h.ptr, n, *args, _PREC[precision], _stream(stream))
    _native.check(rc, 'rve_rom_eval_batch')


def rve_rom_adjoint(h, Fbar, q, gPbar, gFbar, gTheta, status, type=None, stream=None):
    n = Fbar.shape[0]
    g, nm = h.g, h.nmax
    args = [_ptr(type, torch.int32, (n,), 'type') if type is not None else None,
            _ptr(Fbar, torch.float64, (n, g), 'Fbar'), _ptr(q, torch.float64, (n, nm), 'q'),
            _ptr(gPbar, torch.float64, (n, g), 'gPbar'), _ptr(gFbar, torch.float64, (n, g), 'gFbar'),
            _ptr(gTheta, torch.float64, (h.n_types, 2, 2), 'gTheta'),
            _ptr(status, torch.int32, (n,), 'status')]
    _native.check(_native.lib().rve_rom_adjoint(h.ptr, n, *args, _stream(stream)), 'rve_rom_adjoint')


def rve_rom_adjoint_static(h, Fbar, q, gPbar, gFbar, gTheta, status, type=None, stream=None):
    """rve_rom_adjoint without any device allocation in the call, for callers
    that must not allocate (see include/rverom.h): scratch is a static device
    array shared by all calls; overlapping calls race on it."""
    n = Fbar.shape[0]
    g, nm = h.g, h.nmax
    args = [_ptr(type, torch.int32, (n,), 'type') if type is not None else None,
            _ptr(Fbar, torch.float64, (n, g), 'Fbar'), _ptr(q, torch.float64, (n, nm), 'q'),
            _ptr(gPbar, torch.float64, (n, g), 'gPbar'), _ptr(gFbar, torch.float64, (n, g), 'gFbar'),
            _ptr(gTheta, torch.float64, (h.n_types, 2, 2), 'gTheta'),
            _ptr(status, torch.int32, (n,), 'status')]
    _native.check(_native.lib().rve_rom_adjoint_static(h.ptr, n, *args, _stream(stream)),
                  'rve_rom_adjoint_static')


class MeshHandle:
    def __init__(self, ptr, dim, n_nodes, n_elem):
        self.ptr = ptr
        self.dim = dim
        self.g = dim * dim
        self.n_nodes = n_nodes
        self.n_elem = n_elem
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _native.check(_native.lib().macro_mesh_sizes(ptr, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
                      'macro_mesh_sizes')
        self.n_ip, self.n_dof, self.nnz = a.value, b.value, c.value

    def csr(self):
        rp = np.zeros(self.n_dof + 1, dtype=np.int64)
        col = np.zeros(self.nnz, dtype=np.int32)
        _native.check(_native.lib().macro_mesh_csr(self.ptr, rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                                   col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
                      'macro_mesh_csr')
        return rp, col

    def destroy(self):
        if self.ptr:
            _native.check(_native.lib().macro_mesh_destroy(self.ptr), 'macro_mesh_destroy')
            self.ptr = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def macro_mesh_create(X, conn):
    X = np.ascontiguousarray(X, dtype=np.float64)
    conn = np.ascontiguousarray(conn, dtype=np.int64)
    dim = X.shape[1]
    out = ctypes.c_void_p()
    torch.cuda.current_device()
    _native.check(_native.lib().macro_mesh_create(dim, X.shape[0], conn.shape[0],
                                                  X.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                  conn.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                                  ctypes.byref(out)), 'macro_mesh_create')
    return MeshHandle(out, dim, X.shape[0], conn.shape[0])


def macro_gradient(m, u, Fbar, stream=None):
    _native.check(_native.lib().macro_gradient(m.ptr, _ptr(u, torch.float64, (m.n_nodes, m.dim), 'u'),
                                               _ptr(Fbar, torch.float64, (m.n_ip, m.g), 'Fbar'),
                                               _stream(stream)), 'macro_gradient')


def macro_assemble(m, Pbar, dPdF, R, Kvals=None, stream=None):
    _native.check(_native.lib().macro_assemble(
        m.ptr, _ptr(Pbar, torch.float64, (m.n_ip, m.g), 'Pbar'),
        _ptr(dPdF, torch.float64, (m.n_ip, m.g, m.g), 'dPdF') if dPdF is not None else None,
        _ptr(R, torch.float64, (m.n_dof,), 'R'),
        _ptr(Kvals, torch.float64, (m.nnz,), 'Kvals') if Kvals is not None else None,
        _stream(stream)), 'macro_assemble')


def macro_gradient_range(m, e_begin, e_end, u, Fbar, stream=None):
    """Fbar at the integration points of elements e_begin .. e_end - 1 only
    (one shard of a data-parallel macro problem)."""
    n = (e_end - e_begin) * (m.n_ip // m.n_elem)
    _native.check(_native.lib().macro_gradient_range(
        m.ptr, e_begin, e_end, _ptr(u, torch.float64, (m.n_nodes, m.dim), 'u'),
        _ptr(Fbar, torch.float64, (n, m.g), 'Fbar') if n > 0 else None,
        _stream(stream)), 'macro_gradient_range')


def macro_assemble_range(m, e_begin, e_end, Pbar, dPdF, R, Kvals=None, stream=None):
    """Adds the contributions of elements e_begin .. e_end - 1 (their points'
    Pbar and dPdF) to R and Kvals of the whole mesh; zeroes nothing."""
    n = (e_end - e_begin) * (m.n_ip // m.n_elem)
    _native.check(_native.lib().macro_assemble_range(
        m.ptr, e_begin, e_end,
        _ptr(Pbar, torch.float64, (n, m.g), 'Pbar') if n > 0 else None,
        _ptr(dPdF, torch.float64, (n, m.g, m.g), 'dPdF') if (n > 0 and dPdF is not None) else None,
        _ptr(R, torch.float64, (m.n_dof,), 'R'),
        _ptr(Kvals, torch.float64, (m.nnz,), 'Kvals') if Kvals is not None else None,
        _stream(stream)), 'macro_assemble_range')


def macro_residual_norms(m, R, free_mask, rnorm, out, stream=None):
    n = rnorm.shape[0]
    _native.check(_native.lib().macro_residual_norms(
        m.ptr, _ptr(R, torch.float64, (m.n_dof,), 'R'), _ptr(free_mask, torch.uint8, (m.n_dof,), 'free_mask'),
        n, _ptr(rnorm, torch.float64, (n,), 'rnorm'), _ptr(out, torch.float64, (3,), 'out'),
        _stream(stream)), 'macro_residual_norms')


def macro_solve(m, Kvals, R, free_mask, u=None, du=None, info=None, tol=1e-12, max_iter=20000, stream=None):
    """Newton correction of the macro problem on the device: K du = -R on the
    free DOFs (du = 0 on the prescribed ones), u += du when u is given.
    Returns (du, info) with info = [iterations, relative residual, status]
    (device tensors; nothing is synchronized)."""
    n = m.n_dof
    if du is None:
        du = torch.empty(n, dtype=torch.float64, device=R.device)
    if info is None:
        info = torch.empty(3, dtype=torch.float64, device=R.device)
    _native.check(_native.lib().macro_solve(
        m.ptr, _ptr(Kvals, torch.float64, (m.nnz,), 'Kvals'), _ptr(R, torch.float64, (n,), 'R'),
        _ptr(free_mask, torch.uint8, (n,), 'free_mask'), float(tol), int(max_iter),
        _ptr(u, torch.float64, (m.n_nodes, m.dim), 'u') if u is not None else None,
        _ptr(du, torch.float64, (n,), 'du'), _ptr(info, torch.float64, (3,), 'info'), _stream(stream)),
        'macro_solve')
    return du, info


def rve_rom_mmax(h):
    """Largest number of ECM points over the types (history stride)."""
    v = ctypes.c_int32()
    _native.check(_native.lib().rve_rom_mmax(h.ptr, ctypes.byref(v)), 'rve_rom_mmax')
    return v.value


def rve_rom_eval_batch_j2(h, Fbar, q, s, S, Uprev, hist_in, hist_out, plastic, Pbar, dPdF, rnorm, status,
                          type=None, stream=None):
    """rve_rom_eval_batch with small-strain J2 plasticity at the ECM points
    (planar RVEs): plastic [n_types][2][2] = (yield stress, hardening
    modulus) per phase (yield <= 0 or inf: elastic); hist_in / hist_out
    [n][mmax][7] device records (see include/rverom.h)."""
    n = Fbar.shape[0]
    g, ns, nm = h.g, h.ns, h.nmax
    mm = rve_rom_mmax(h)
    pl = np.ascontiguousarray(plastic, dtype=np.float64).reshape(h.n_types * 4)
    args = [_ptr(type, torch.int32, (n,), 'type') if type is not None else None,
            _ptr(Fbar, torch.float64, (n, g), 'Fbar'),
            _ptr(q, torch.float64, (n, nm), 'q'), _ptr(s, torch.float64, (n, nm), 's'),
            _ptr(S, torch.float64, (n, nm, ns), 'S'), _ptr(Uprev, torch.float64, (n, ns), 'Uprev'),
            _ptr(hist_in, torch.float64, (n, mm, 7), 'hist_in'), _ptr(hist_out, torch.float64, (n, mm, 7), 'hist_out'),
            pl.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            _ptr(Pbar, torch.float64, (n, g), 'Pbar'), _ptr(dPdF, torch.float64, (n, g, g), 'dPdF'),
            _ptr(rnorm, torch.float64, (n,), 'rnorm'), _ptr(status, torch.int32, (n,), 'status')]
    _native.check(_native.lib().rve_rom_eval_batch_j2(h.ptr, n, *args, _stream(stream)), 'rve_rom_eval_batch_j2')


def rve_rom_biot_cauchy(Fbar, Pbar, dPdF, biot=None, cbiot=None, sigma=None, csigma=None, stream=None):
    """Biot stress and tangent, Cauchy stress and its approximate tangent of
    every point (Sec. 3.2.2, Appendix A); returns the four output tensors."""
    n, g = Fbar.shape
    dim = 2 if g == 4 else 3
    ns = 3 if dim == 2 else 6
    dev = Fbar.device
    mk = lambda x, shp: torch.empty(shp, dtype=torch.float64, device=dev) if x is None else x
    biot, sigma = mk(biot, (n, ns)), mk(sigma, (n, ns))
    cbiot, csigma = mk(cbiot, (n, ns, ns)), mk(csigma, (n, ns, ns))
    _native.check(_native.lib().rve_rom_biot_cauchy(
        dim, n, _ptr(Fbar, torch.float64, (n, g), 'Fbar'), _ptr(Pbar, torch.float64, (n, g), 'Pbar'),
        _ptr(dPdF, torch.float64, (n, g, g), 'dPdF'), _ptr(biot, torch.float64, (n, ns), 'biot'),
        _ptr(cbiot, torch.float64, (n, ns, ns), 'cbiot'), _ptr(sigma, torch.float64, (n, ns), 'sigma'),
        _ptr(csigma, torch.float64, (n, ns, ns), 'csigma'), _stream(stream)), 'rve_rom_biot_cauchy')
    return biot, cbiot, sigma, csigma


def surrogate_linear_eval(C0, Fbar, Pbar, dPdF=None, stream=None):
    """Linear-elastic surrogate Pbar = C0 (Fbar - I), dPdF = C0 (Box 2, step 1)."""
    n, g = Fbar.shape
    _native.check(_native.lib().surrogate_linear_eval(
        2 if g == 4 else 3, n, _ptr(C0, torch.float64, (g, g), 'C0'), _ptr(Fbar, torch.float64, (n, g), 'Fbar'),
        _ptr(Pbar, torch.float64, (n, g), 'Pbar'),
        _ptr(dPdF, torch.float64, (n, g, g), 'dPdF') if dPdF is not None else None, _stream(stream)),
        'surrogate_linear_eval')


def paths_kmeans(X, centers, max_iter=200, labels=None, stream=None):
    """k-means of the rows of X (device [n][dim]) from the given centres
    (updated in place); returns (labels, updates done, inertia)."""
    n, dim = X.shape
    k = centers.shape[0]
    if labels is None:
        labels = torch.empty(n, dtype=torch.int32, device=X.device)
    info = (ctypes.c_double * 2)()
    _native.check(_native.lib().paths_kmeans(
        n, dim, _ptr(X, torch.float64, (n, dim), 'X'), k, _ptr(centers, torch.float64, (k, dim), 'centers'),
        _ptr(labels, torch.int32, (n,), 'labels'), int(max_iter), info, _stream(stream)), 'paths_kmeans')
    return labels, int(info[0]), info[1]


def rverom_df_log(x, out, stream=None):
    """The library's double-float logarithm at the points of x (float64, CUDA)."""
    n = x.shape[0]
    _native.check(_native.lib().rverom_df_log(n, _ptr(x, torch.float64, (n,), 'x'),
                                              _ptr(out, torch.float64, (n,), 'out'), _stream(stream)),
                  'rverom_df_log')


PEAK_UNITS = {'fp32': 0, 'fp64': 1, 'tf32': 2, 'bf16': 3}


def rverom_peak_probe(unit, stream=None):
    """Measured TFLOP/s of one execution unit ('fp32', 'fp64', 'tf32' or
    'bf16') of the current device."""
    v = ctypes.c_double()
    _native.check(_native.lib().rverom_peak_probe(PEAK_UNITS[unit], ctypes.byref(v), _stream(stream)),
                  'rverom_peak_probe')
    return v.value
