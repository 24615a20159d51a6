"""rve_rom_adjoint_static, the allocation-free variant of the adjoint, for
callers that must not allocate device memory during the call (for example
a macro FE code calling it from per-increment material callbacks, where an
allocation may synchronize the device, or a process whose device memory is
reserved by another allocator).  Its results must equal those of
rve_rom_adjoint on two calls in a row (the static scratch keeps the previous
call's contents, so the second call checks that nothing leaks between calls).
Collected last so that a failure here never hides the other GPU tests."""
import os

import numpy as np
import pytest
import torch

import synthetic as syn
from conftest import rom_path

pytestmark = pytest.mark.gpu
rv = pytest.importorskip('paper_2306_02687_gb300')


def _handle(names):
    roms = [rv.load_rom_file(rom_path(nm)) for nm in names]
    return rv.rve_rom_create(2, roms, roms[0]['V0'])


def _inputs(h, n, seed, types=None, nmodes=None):
    F = syn.fbar_batch(seed, 2, n, 0.1, 0.3).reshape(n, 4)
    q = np.zeros((n, h.nmax))
    for a in range(n):
        k = h.nmax if nmodes is None else nmodes[types[a]]
        q[a, :k] = syn.perturbation(seed + 1 + a, k, 1e-3)
    gP = syn.perturbation(seed + 999, (n, 4), 1.0)
    T = lambda x: torch.tensor(x, dtype=torch.float64, device='cuda')
    return T(F), T(q), T(gP)


def _run(fn, h, F, q, gP, types):
    n = F.shape[0]
    gF = torch.empty(n, 4, dtype=torch.float64, device='cuda')
    gth = torch.zeros(h.n_types, 2, 2, dtype=torch.float64, device='cuda')
    st = torch.empty(n, dtype=torch.int32, device='cuda')
    fn(h, F, q, gP, gF, gth, st, type=types)
    torch.cuda.synchronize()
    return gF.cpu().numpy(), gth.cpu().numpy(), st.cpu().numpy()


def _close(a, b, tol):
    return np.abs(a - b).max() <= tol * max(np.abs(b).max(), 1e-300)


def test_static_adjoint_matches_allocating_adjoint():
    h = _handle(['c1'])
    F, q, gP = _inputs(h, 37, syn.SEED_BASE + 60)
    ref = _run(rv.rve_rom_adjoint, h, F, q, gP, None)
    for _ in range(2):
        got = _run(rv.rve_rom_adjoint_static, h, F, q, gP, None)
        assert np.all(got[2] == 0) and np.all(ref[2] == 0)
        assert _close(got[0], ref[0], 1e-12) and _close(got[1], ref[1], 1e-12)


def test_static_adjoint_mixed_types_and_limit():
    names = ['c5a', 'c5b', 'c5c']
    if not all(os.path.exists(rom_path(nm)) for nm in names):
        pytest.skip('mixed-type ROM files not generated')
    h = _handle(names)
    n = 30
    types_np = syn.type_labels(syn.SEED_BASE + 61, n, 3)
    nmodes = [16, 32, 64]
    F, q, gP = _inputs(h, n, syn.SEED_BASE + 62, types_np, nmodes)
    types = torch.tensor(types_np, device='cuda')
    ref = _run(rv.rve_rom_adjoint, h, F, q, gP, types)
    for _ in range(2):
        got = _run(rv.rve_rom_adjoint_static, h, F, q, gP, types)
        assert np.all(got[2] == ref[2])
        assert _close(got[0], ref[0], 1e-12) and _close(got[1], ref[1], 1e-12)
    # a typed batch beyond the static point-list capacity is refused before any work
    big = (1 << 20) + 1
    Fb = torch.zeros(big, 4, dtype=torch.float64, device='cuda')
    qb = torch.zeros(big, h.nmax, dtype=torch.float64, device='cuda')
    tb = torch.zeros(big, dtype=torch.int32, device='cuda')
    gb = torch.zeros(big, 4, dtype=torch.float64, device='cuda')
    with pytest.raises(RuntimeError, match='SCRATCH_LIMIT'):
        rv.rve_rom_adjoint_static(h, Fb, qb, gb, torch.empty_like(gb),
                                  torch.zeros(3, 2, 2, dtype=torch.float64, device='cuda'),
                                  torch.empty(big, dtype=torch.int32, device='cuda'), type=tb)
