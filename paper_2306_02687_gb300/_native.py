"""ctypes loader of librverom.so (argument marshalling only).

The library must have been built in-tree (paper_2306_02687_gb300.build); there
is no fallback of any kind: a missing library raises at first use.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, 'librverom.so')

c_int = ctypes.c_int32
c_i64 = ctypes.c_int64
c_dbl = ctypes.c_double
c_vp = ctypes.c_void_p
P = ctypes.POINTER


class TypeDesc(ctypes.Structure):
    _fields_ = [('n_modes', ctypes.c_int32), ('n_ecm', ctypes.c_int32),
                ('B', P(c_dbl)), ('w', P(c_dbl)), ('phase', P(ctypes.c_int32)),
                ('moduli', (c_dbl * 2) * 2)]


# name -> (restype, argtypes); every entry point declared in include/rverom.h
SIGNATURES = {
    'rve_rom_create': (c_int, [c_int, c_int, P(TypeDesc), c_dbl, P(c_vp)]),
    'rve_rom_destroy': (c_int, [c_vp]),
    'rve_rom_set_moduli': (c_int, [c_vp, c_int, P(c_dbl)]),
    'rve_rom_nmax': (c_int, [c_vp, P(c_int)]),
    'rve_rom_autotune': (c_int, [c_vp, c_int, c_i64, P(ctypes.c_float), c_vp]),
    'rve_rom_select_kernel': (c_int, [c_vp, c_int, c_int, c_int, P(c_int)]),
    'rve_rom_kernel_info': (c_int, [c_vp, c_int, c_int, c_int, ctypes.c_char_p, c_int, P(c_int)]),
    'rve_rom_eval_batch': (c_int, [c_vp, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp,
                                   c_vp, c_vp, c_int, c_vp]),
    'rve_rom_adjoint': (c_int, [c_vp, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    'rve_rom_adjoint_static': (c_int, [c_vp, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    'macro_mesh_create': (c_int, [c_int, c_i64, c_i64, P(c_dbl), P(c_i64), P(c_vp)]),
    'macro_mesh_destroy': (c_int, [c_vp]),
    'macro_mesh_sizes': (c_int, [c_vp, P(c_i64), P(c_i64), P(c_i64)]),
    'macro_mesh_csr': (c_int, [c_vp, P(c_i64), P(c_int)]),
    'macro_gradient': (c_int, [c_vp, c_vp, c_vp, c_vp]),
    'macro_assemble': (c_int, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    'macro_gradient_range': (c_int, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp]),
    'macro_assemble_range': (c_int, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp]),
    'macro_residual_norms': (c_int, [c_vp, c_vp, c_vp, c_i64, c_vp, c_vp, c_vp]),
    'macro_solve': (c_int, [c_vp, c_vp, c_vp, c_vp, c_dbl, c_int, c_vp, c_vp, c_vp, c_vp]),
    'rve_rom_mmax': (c_int, [c_vp, P(c_int)]),
    'rve_rom_eval_batch_j2': (c_int, [c_vp, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp,
                                      P(c_dbl), c_vp, c_vp, c_vp, c_vp, c_vp]),
    'rve_snapshots': (c_int, [c_int, c_vp, P(c_dbl), c_int, c_int, c_vp, c_int, c_dbl, c_dbl, c_int, c_int,
                              c_vp, c_vp, c_vp]),
    'pod_modes': (c_int, [c_i64, c_int, c_vp, c_int, c_vp, c_int, c_vp, c_vp, c_vp, c_vp]),
    'rve_mode_gradients': (c_int, [c_int, c_int, c_vp, c_vp, c_vp]),
    'ecm_training_matrix': (c_int, [c_int, c_vp, P(c_dbl), c_int, c_vp, c_int, c_vp, c_vp, c_vp, c_vp]),
    'ecm_select': (c_int, [c_i64, c_int, c_vp, c_dbl, c_int, c_vp, c_int, c_int, c_vp, c_vp, P(c_int), P(c_dbl),
                           c_vp]),
    'rve_rom_biot_cauchy': (c_int, [c_int, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    'surrogate_linear_eval': (c_int, [c_int, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp]),
    'paths_kmeans': (c_int, [c_i64, c_int, c_vp, c_int, c_vp, c_vp, c_int, P(c_dbl), c_vp]),
    'rverom_df_log': (c_int, [c_i64, c_vp, c_vp, c_vp]),
    'rverom_peak_probe': (c_int, [c_int, P(c_dbl), c_vp]),
}

_lib = None


def lib():
    """Load the native library once; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError('librverom.so is missing: build it with '
                               'python -m paper_2306_02687_gb300.build (no CPU fallback exists)')
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


ERRORS = {-1: 'RVEROM_ERR_ARG', -2: 'RVEROM_ERR_CUDA', -3: 'RVEROM_ERR_UNSUPPORTED',
          -4: 'RVEROM_ERR_SCRATCH_LIMIT (batch larger than the static scratch of rve_rom_adjoint_static)'}


def check(rc, what):
    if rc != 0:
        raise RuntimeError('%s failed: %s (%d)' % (what, ERRORS.get(rc, '?'), rc))
