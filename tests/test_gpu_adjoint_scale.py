"""The implicit adjoint at the size of the differentiation workload (the
16x16 / 12-mode / 60-point ROM at 16384 macro points, the launch the
benchmark times): sampled points against the oracle's adjoint, the
moduli cotangent against central finite differences of the GPU's converged
stresses (h = 1e-6, float64), and the Fbar cotangent against central
differences along a random direction per point."""
import numpy as np
import pytest
import torch

import synthetic as syn
from conftest import rom_path
from oracle import adjoint, reduced

pytestmark = pytest.mark.gpu
rv = pytest.importorskip('paper_2306_02687_gb300')

N = 16384


def T(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device='cuda')


def _converged(h, Fd, iters=14):
    q, s, S, U = h.zero_state(Fd.shape[0])
    Pbar, dPdF, rnorm, status = h.outputs(Fd.shape[0])
    for _ in range(iters):
        rv.rve_rom_eval_batch(h, Fd, q, s, S, U, Pbar, dPdF, rnorm, status, precision='fp64')
    torch.cuda.synchronize()
    assert status.max().item() == 0 and rnorm.max().item() < 1e-12
    return q, Pbar


@pytest.fixture(scope='module')
def setup():
    roms = [rv.load_rom_file(rom_path('c1'))]
    h = rv.rve_rom_create(2, roms, roms[0]['V0'])
    orom = reduced.Rom.load(rom_path('c1'))
    F = syn.fbar_batch(syn.SEED_BASE + 90, 2, N, 0.1, 0.3)
    Fd = T(F.reshape(N, 4))
    q, Pbar = _converged(h, Fd)
    gP = syn.perturbation(syn.SEED_BASE + 91, (N, 4), 1.0)
    return h, orom, F, Fd, q, Pbar, gP


def test_adjoint_full_size_sampled_against_oracle(setup):
    h, orom, F, Fd, q, Pbar, gP = setup
    idx = np.sort(syn.rng(92).choice(N, 32, replace=False))
    # the sampled points carry the oracle's converged states (oracle inputs
    # only); the cotangent is zero elsewhere, so that gTheta sums the sample
    qs = q.clone()
    for a in idx:
        o, _ = reduced.converge_point(orom, F[a], tol=1e-14 * orom.moduli[0, 0])
        qs[a] = T(o['q'])
    gPs = np.zeros_like(gP)
    gPs[idx] = gP[idx]
    gF = torch.empty(N, 4, dtype=torch.float64, device='cuda')
    gth = torch.zeros(1, 2, 2, dtype=torch.float64, device='cuda')
    st = torch.empty(N, dtype=torch.int32, device='cuda')
    rv.rve_rom_adjoint(h, Fd, qs, T(gPs), gF, gth, st)
    torch.cuda.synchronize()
    assert st.max().item() == 0
    gFh = gF.cpu().numpy()
    ref = np.zeros((2, 2))
    for a in idx:
        gf, gt = adjoint.point_adjoint(orom, F[a], qs[a].cpu().numpy(), gP[a])
        assert np.abs(gFh[a] - gf).max() <= 1e-11 * np.abs(gf).max()
        ref += gt
    assert np.abs(gth.cpu().numpy()[0] - ref).max() <= 1e-10 * np.abs(ref).max()
    assert np.all(gFh[np.setdiff1d(np.arange(N), idx)] == 0.0)


def test_adjoint_full_size_against_finite_differences(setup):
    h, orom, F, Fd, q, Pbar, gP = setup
    gPd = T(gP)
    gF = torch.empty(N, 4, dtype=torch.float64, device='cuda')
    gth = torch.zeros(1, 2, 2, dtype=torch.float64, device='cuda')
    st = torch.empty(N, dtype=torch.int32, device='cuda')
    rv.rve_rom_adjoint(h, Fd, q, gPd, gF, gth, st)
    torch.cuda.synchronize()
    assert st.max().item() == 0
    got = gth.cpu().numpy()[0]
    hh = 1e-6
    mod = orom.moduli.copy()
    # moduli: d/dtheta of sum_alpha <gP_alpha, Pbar_alpha> at converged states
    for ph in range(2):
        for k in range(2):
            vals = []
            for sgn in (1.0, -1.0):
                m2 = mod.copy()
                m2[ph, k] += sgn * hh
                rv.rve_rom_set_moduli(h, 0, m2)
                _, P2 = _converged(h, Fd)
                vals.append((P2 * gPd).sum().item())
            rv.rve_rom_set_moduli(h, 0, mod)
            fd = (vals[0] - vals[1]) / (2 * hh)
            print('theta', ph, k, got[ph, k], fd)
            assert abs(fd - got[ph, k]) <= 1e-6 * np.abs(got).max()
    # Fbar: along a random direction V per point, d<gP, Pbar(F + t V)>/dt = <gF, V>
    V = T(syn.perturbation(syn.SEED_BASE + 93, (N, 4), 1.0))
    vals = []
    for sgn in (1.0, -1.0):
        _, P2 = _converged(h, Fd + sgn * hh * V)
        vals.append((P2 * gPd).sum(dim=1))
    fd = ((vals[0] - vals[1]) / (2 * hh)).cpu().numpy()
    an = (gF * V).sum(dim=1).cpu().numpy()
    scale = np.abs(an).max()
    print('Fbar directional: max abs diff %.3e of %.3e' % (np.abs(fd - an).max(), scale))
    assert np.abs(fd - an).max() <= 1e-6 * scale
