"""Plain C++ float64 CPU baseline of the batched hyper-reduced RVE evaluation
(steps a1-a7), OpenMP over macro points: the host-core timing baseline of the
benchmark.  It shares no code with the CUDA library (paper_2306_02687_gb300)
or the test oracle (oracle/); the tests pin it against the oracle.

  build()                 compile librom_cpu.so in this directory (g++ -O3 -fopenmp)
  eval_batch(rom, ...)    evaluate a batch of one RVE type on n threads
"""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, 'rom_eval_cpu.cpp')
LIB = os.path.join(HERE, 'librom_cpu.so')
_lib = None


def build():
    tmp = LIB + '.tmp'
    cmd = ['g++', '-O3', '-std=c++17', '-fopenmp', '-fPIC', '-shared', SRC, '-o', tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError('g++ failed:\n%s\n%s' % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            build()
        L = ctypes.CDLL(LIB)
        vp = ctypes.c_void_p
        L.rom_eval_cpu.restype = ctypes.c_int
        L.rom_eval_cpu.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, ctypes.c_double,
                                   ctypes.c_int64, vp, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_int]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def eval_batch(rom, Fbar, q, s, S, Uprev, nthreads=0):
    """rom: dict(B [m][g][n], w, phase, moduli [2][2], V0).  Fbar [N][g];
    state arrays (float64, unpadded, updated in place): q, s [N][n],
    S [N][n][ns], Uprev [N][ns].  Returns (dict of outputs, threads used)."""
    B = np.ascontiguousarray(rom['B'], dtype=np.float64)
    m, g, n = B.shape
    d = int(round(np.sqrt(g)))
    w = np.ascontiguousarray(rom['w'], dtype=np.float64)
    ph = np.ascontiguousarray(rom['phase'], dtype=np.int32)
    mod = np.ascontiguousarray(rom['moduli'], dtype=np.float64).reshape(4)
    N = len(Fbar)
    F = np.ascontiguousarray(Fbar, dtype=np.float64).reshape(N, g)
    for x in (q, s, S, Uprev):
        assert x.dtype == np.float64 and x.flags['C_CONTIGUOUS']
    Pbar = np.empty((N, g))
    dPdF = np.empty((N, g, g))
    rnorm = np.empty(N)
    status = np.empty(N, dtype=np.int32)
    used = lib().rom_eval_cpu(d, n, m, _p(B), _p(w), _p(ph), _p(mod), float(rom['V0']), N, _p(F), _p(q), _p(s),
                              _p(S), _p(Uprev), _p(Pbar), _p(dPdF), _p(rnorm), _p(status), int(nthreads))
    return dict(Pbar=Pbar, dPdF=dPdF, rnorm=rnorm, status=status, q=q, s=s, S=S, Uprev=Uprev), used
