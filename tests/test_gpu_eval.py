"""GPU parity of rve_rom_eval_batch (through the C ABI) against the CPU
oracle, element by element on identical seeded inputs."""
import numpy as np
import pytest
import torch

import synthetic as syn
from conftest import rom_path
from oracle import reduced, polar

pytestmark = pytest.mark.gpu

rv = pytest.importorskip('paper_2306_02687_gb300')


def _handle(names):
    roms = [rv.load_rom_file(rom_path(nm)) for nm in names]
    d = int(round(np.sqrt(roms[0]['B'].shape[1])))
    return rv.rve_rom_create(d, roms, roms[0]['V0']), [reduced.Rom.load(rom_path(nm)) for nm in names]


@pytest.fixture(scope='module')
def c1():
    return _handle(['c1'])


def converged_states(orom, F, pert, seed):
    """Oracle-converged q at each F plus a seeded relative perturbation."""
    n = len(F)
    qs = np.zeros((n, orom.n))
    for a in range(n):
        o, _ = reduced.converge_point(orom, F[a])
        qs[a] = o['q'] + syn.perturbation(seed + a, orom.n, pert * np.abs(o['q']).max())
    return qs


def run_gpu(h, F, q, s, S, U, precision, types=None):
    n = len(F)
    dev = 'cuda'
    t = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=dev)
    Fd, qd, sd, Sd, Ud = t(F.reshape(n, -1)), t(q), t(s), t(S), t(U)
    Pbar, dPdF, rnorm, status = h.outputs(n)
    ty = None if types is None else torch.tensor(types, dtype=torch.int32, device=dev)
    rv.rve_rom_eval_batch(h, Fd, qd, sd, Sd, Ud, Pbar, dPdF, rnorm, status, type=ty, precision=precision)
    torch.cuda.synchronize()
    c = lambda x: x.cpu().numpy()
    return dict(Pbar=c(Pbar), dPdF=c(dPdF), rnorm=c(rnorm), status=c(status), q=c(qd), s=c(sd), S=c(Sd),
                Uprev=c(Ud))


def pad(x, nmax):
    out = np.zeros((nmax,) + x.shape[1:])
    out[:x.shape[0]] = x
    return out


def oracle_batch(oroms, F, q, s, S, U, types=None):
    outs = []
    for a in range(len(F)):
        r = oroms[0 if types is None else types[a]]
        n = r.n
        outs.append(reduced.eval_point(r, F[a], q[a][:n], s[a][:n], S[a][:n], U[a]))
    return outs


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def compare(g, outs, nmax, tol):
    errs = dict(Pbar=0.0, dPdF=0.0, s=0.0, S=0.0, q=0.0, rnorm=0.0, Uprev=0.0)
    for a, o in enumerate(outs):
        assert g['status'][a] == o['status'] == 0
        n = len(o['q'])
        errs['Pbar'] = max(errs['Pbar'], rel(g['Pbar'][a], o['Pbar'].ravel()))
        errs['dPdF'] = max(errs['dPdF'], rel(g['dPdF'][a], o['dPdF']))
        errs['s'] = max(errs['s'], rel(g['s'][a][:n], o['s']))
        errs['S'] = max(errs['S'], rel(g['S'][a][:n], o['S']))
        errs['q'] = max(errs['q'], rel(g['q'][a][:n], o['q']))
        errs['Uprev'] = max(errs['Uprev'], rel(g['Uprev'][a], o['Uprev']))
        errs['rnorm'] = max(errs['rnorm'], abs(g['rnorm'][a] - o['rnorm']) / max(o['rnorm'], 1e-300))
        assert np.all(g['q'][a][n:] == 0) and np.all(g['s'][a][n:] == 0)
    print({k: '%.2e' % v for k, v in errs.items()})
    for k, v in tol.items():
        assert errs[k] <= v, (k, errs[k], v)
    return errs


def mid_newton_inputs(orom, n, seed, eps=0.1, angle=0.3):
    """States of a monolithic iteration: converged at F0, evaluated at a
    nearby F1 with the stored s, S, Uprev, plus a perturbation of q."""
    F0 = syn.fbar_batch(seed, orom.d, n, eps, angle)
    dF = syn.perturbation(seed + 1, F0.shape, 2e-3)
    F1 = F0 + dF
    nmax = orom.n
    q = np.zeros((n, nmax))
    s = np.zeros((n, nmax))
    S = np.zeros((n, nmax, orom.ns))
    U = np.zeros((n, orom.ns))
    for a in range(n):
        o, _ = reduced.converge_point(orom, F0[a])
        q[a] = o['q'] + syn.perturbation(seed + 7 + a, nmax, 1e-3 * np.abs(o['q']).max())
        s[a], S[a], U[a] = o['s'], o['S'], o['Uprev']
    return F1, q, s, S, U


# FP64 form: the same float64 arithmetic in another summation order.  Uprev
# is the polar stretch, computed by Newton iteration on the GPU and by an
# eigen-decomposition in the oracle (3D): a few units of rounding apart.
TOL_FP64 = dict(Pbar=1e-12, dPdF=1e-11, s=1e-9, S=1e-9, q=1e-12, Uprev=1e-14, rnorm=1e-9)
# mixed form on mid-Newton states: FP64 r and Pbar_U; the Newton correction
# K_qF^T K^-1 r carries the float32 solve error (small near convergence)
TOL_MIXED = dict(Pbar=1e-8, dPdF=1e-5, q=1e-12, Uprev=1e-14, rnorm=1e-6)


@pytest.mark.parametrize('n', [1, 15, 37])
def test_fp64_fresh_state(c1, n):
    h, oroms = c1
    F = syn.fbar_batch(syn.SEED_BASE + 11, 2, n, 0.1, 0.3)
    q, s, S, U = (np.zeros((n, h.nmax)), np.zeros((n, h.nmax)), np.zeros((n, h.nmax, 3)),
                  np.tile([1.0, 1.0, 0.0], (n, 1)))
    g = run_gpu(h, F, q, s, S, U, 'fp64')
    compare(g, oracle_batch(oroms, F, q, s, S, U), h.nmax, TOL_FP64)


def test_fp64_mid_newton(c1):
    h, oroms = c1
    F, q, s, S, U = mid_newton_inputs(oroms[0], 40, syn.SEED_BASE + 12)
    g = run_gpu(h, F, q, s, S, U, 'fp64')
    compare(g, oracle_batch(oroms, F, q, s, S, U), h.nmax, TOL_FP64)


def test_mixed_mid_newton(c1):
    h, oroms = c1
    F, q, s, S, U = mid_newton_inputs(oroms[0], 40, syn.SEED_BASE + 13)
    g = run_gpu(h, F, q, s, S, U, 'mixed')
    compare(g, oracle_batch(oroms, F, q, s, S, U), h.nmax, TOL_MIXED)


@pytest.mark.parametrize('precision', ['fp64', 'mixed'])
def test_converged_stress_matches_oracle(c1, precision):
    # Newton as iterative refinement: at convergence both forms meet the
    # float64 oracle's converged stress
    h, oroms = c1
    n = 24
    F = syn.fbar_batch(syn.SEED_BASE + 14, 2, n, 0.1, 0.5)
    dev = 'cuda'
    Fd = torch.tensor(F.reshape(n, 4), device=dev)
    q, s, S, U = h.zero_state(n)
    Pbar, dPdF, rnorm, status = h.outputs(n)
    for it in range(12):
        rv.rve_rom_eval_batch(h, Fd, q, s, S, U, Pbar, dPdF, rnorm, status, precision=precision)
    torch.cuda.synchronize()
    assert rnorm.max().item() < 1e-12 and status.max().item() == 0
    P = Pbar.cpu().numpy()
    C = dPdF.cpu().numpy()
    for a in range(n):
        o, _ = reduced.converge_point(oroms[0], F[a])
        assert rel(P[a], o['Pbar'].ravel()) <= 1e-10
        assert rel(C[a], o['dPdF']) <= (1e-10 if precision == 'fp64' else 1e-5)


def each_candidate(h, precision):
    """Select every compiled forward candidate of type 0 in turn."""
    nc = rv.rve_rom_select_kernel(h, 0, precision)
    for c in range(nc):
        rv.rve_rom_select_kernel(h, 0, precision, c)
        yield c
    rv.rve_rom_select_kernel(h, 0, precision, 0)


@pytest.mark.parametrize('precision', ['fp64', 'mixed'])
def test_status_codes_and_empty_batch(c1, precision):
    # every candidate (SIMT and tensor-core forms) reports the same statuses,
    # NaN outputs for failed points and leaves their micro state untouched
    h, oroms = c1
    n = 5
    F = syn.fbar_batch(syn.SEED_BASE + 15, 2, n, 0.1, 0.3)
    F[1] = np.array([[-1.0, 0.0], [0.0, 1.0]])           # det F <= 0
    F[3, 0, 0] = np.nan                                  # non-finite input
    q, s, S, U = (np.zeros((n, h.nmax)), np.zeros((n, h.nmax)), np.zeros((n, h.nmax, 3)),
                  np.tile([1.0, 1.0, 0.0], (n, 1)))
    q2 = q.copy()
    q2[0] = 50.0
    o2 = reduced.eval_point(oroms[0], F[0], q2[0], s[0], S[0], U[0])
    for _ in each_candidate(h, precision):
        g = run_gpu(h, F, q, s, S, U, precision)
        assert list(g['status']) == [0, 1, 0, 3, 0]
        assert np.all(np.isnan(g['Pbar'][[1, 3]])) and np.all(np.isnan(g['dPdF'][[1, 3]]))
        assert np.all(np.isfinite(g['Pbar'][[0, 2, 4]]))
        # micro det F <= 0: a huge fluctuation amplitude folds some ECM point
        g2 = run_gpu(h, F[[0]], q2[[0]], s[[0]], S[[0]], U[[0]], precision)
        assert g2['status'][0] == o2['status'] == 1
        assert np.array_equal(g2['q'][0], q2[0]) and np.array_equal(g2['Uprev'][0], U[0])
    # empty batch is a no-op
    z = torch.zeros(0, 4, dtype=torch.float64, device='cuda')
    qz, sz, Sz, Uz = h.zero_state(0)
    Pz, dz, rz, stz = h.outputs(0)
    rv.rve_rom_eval_batch(h, z, qz, sz, Sz, Uz, Pz, dz, rz, stz)


@pytest.mark.parametrize('precision', ['fp64', 'mixed'])
def test_nonspd_reduced_stiffness(precision):
    h, oroms = _handle(['c1'])
    mod = oroms[0].moduli.copy()
    mod[:, 0] = -0.3                                     # negative shear modulus
    rv.rve_rom_set_moduli(h, 0, mod)
    n = 3
    F = syn.fbar_batch(syn.SEED_BASE + 16, 2, n, 0.05, 0.0)
    q, s, S, U = (np.zeros((n, h.nmax)), np.zeros((n, h.nmax)), np.zeros((n, h.nmax, 3)),
                  np.tile([1.0, 1.0, 0.0], (n, 1)))
    r = oroms[0].with_moduli(mod)
    outs = [reduced.eval_point(r, F[a], q[a], s[a], S[a], U[a]) for a in range(n)]
    for _ in each_candidate(h, precision):
        g = run_gpu(h, F, q, s, S, U, precision)
        for a in range(n):
            assert g['status'][a] == outs[a]['status'] == 2
        assert np.all(np.isnan(g['Pbar']))


def test_full_size_2d_sampled():
    # 48x48 RVE / 24 modes / 200 ECM points at 16384 macro points (the
    # benchmark's launch configuration); 32 sampled points carry oracle
    # mid-Newton states and are compared with the oracle one by one, under
    # the default candidate and under the autotuner's pick
    h, oroms = _handle(['c2'])
    n = 16384
    orom = oroms[0]
    idx = np.sort(syn.rng(5).choice(n, 32, replace=False))
    F = syn.fbar_batch(syn.SEED_BASE + 2, 2, n, 0.15, 0.3)
    q = np.zeros((n, h.nmax))
    s = np.zeros((n, h.nmax))
    S = np.zeros((n, h.nmax, 3))
    U = np.tile([1.0, 1.0, 0.0], (n, 1))
    Fm, qm, sm, Sm, Um = mid_newton_inputs(orom, len(idx), syn.SEED_BASE + 21, eps=0.15)
    F[idx], q[idx], s[idx], S[idx], U[idx] = Fm, qm, sm, Sm, Um
    outs = oracle_batch(oroms, F[idx], q[idx], s[idx], S[idx], U[idx])
    for precision, tol in (('fp64', TOL_FP64), ('mixed', TOL_MIXED)):
        g = run_gpu(h, F, q, s, S, U, precision)
        assert np.all(g['status'] == 0)
        compare({k: v[idx] for k, v in g.items()}, outs, h.nmax, tol)
        # the autotuner's pick (the benchmark's kernel) on the same batch
        ms = rv.rve_rom_autotune(h, precision, n_sample=n)
        assert np.all(ms[0][ms[0] != -1] > 0), ms      # no candidate rejected for a bad status
        g = run_gpu(h, F, q, s, S, U, precision)
        assert np.all(g['status'] == 0)
        print(precision, 'autotuned:', rv.rve_rom_kernel_info(h, 0, precision)[0])
        compare({k: v[idx] for k, v in g.items()}, outs, h.nmax, tol)


def test_mixed_error_is_a_fraction_of_the_newton_correction(c1):
    # far from equilibrium (fresh state at 10% stretch) the mixed-form error
    # of Pbar_alg is bounded by a small multiple of eps32 * cond(K) times the
    # correction |Pbar_U - Pbar_alg|; the converged result is float64-exact
    h, oroms = c1
    n = 32
    F = syn.fbar_batch(syn.SEED_BASE + 22, 2, n, 0.1, 0.3)
    q, s, S, U = (np.zeros((n, h.nmax)), np.zeros((n, h.nmax)), np.zeros((n, h.nmax, 3)),
                  np.tile([1.0, 1.0, 0.0], (n, 1)))
    g = run_gpu(h, F, q, s, S, U, 'mixed')
    for a, o in enumerate(oracle_batch(oroms, F, q, s, S, U)):
        R, Uu = polar.polar(F[a])
        PU = reduced.reduced_system(oroms[0], Uu, q[a])[1].reshape(2, 2) / oroms[0].V0
        corr = np.abs(R @ PU - o['Pbar']).max()
        assert np.abs(g['Pbar'][a] - o['Pbar'].ravel()).max() <= 1e-4 * corr


def test_mixed_types_batch():
    names = ['c5a', 'c5b', 'c5c']
    import os
    if not all(os.path.exists(rom_path(nm)) for nm in names):
        pytest.skip('mixed-type ROM files not generated')
    h, oroms = _handle(names)
    n = 45
    types = syn.type_labels(syn.SEED_BASE + 17, n, 3)
    F = syn.fbar_batch(syn.SEED_BASE + 18, 2, n, 0.14, 0.3)
    q = np.zeros((n, h.nmax))
    s = np.zeros((n, h.nmax))
    S = np.zeros((n, h.nmax, 3))
    U = np.zeros((n, 3))
    for t in range(3):
        sel = np.nonzero(types == t)[0]
        Fm, qm, sm, Sm, Um = mid_newton_inputs(oroms[t], len(sel), syn.SEED_BASE + 30 + t, eps=0.14)
        nt = oroms[t].n
        F[sel], q[sel, :nt], s[sel, :nt], S[sel, :nt], U[sel] = Fm, qm, sm, Sm, Um
    for precision, tol in (('fp64', TOL_FP64), ('mixed', TOL_MIXED)):
        g = run_gpu(h, F, q, s, S, U, precision, types=types)
        compare(g, oracle_batch(oroms, F, q, s, S, U, types), h.nmax, tol)
    bad = types.copy()
    bad[4] = 7
    g = run_gpu(h, F, q, s, S, U, 'fp64', types=bad)
    assert g['status'][4] == 3 and np.all(g['status'][np.arange(n) != 4] == 0)


def test_3d_batch():
    import os
    if not os.path.exists(rom_path('c3')):
        pytest.skip('3D ROM file not generated')
    h, oroms = _handle(['c3'])
    n = 9
    F, q, s, S, U = mid_newton_inputs(oroms[0], n, syn.SEED_BASE + 20, eps=0.2, angle=0.4)
    outs = oracle_batch(oroms, F, q, s, S, U)
    for precision, tol in (('fp64', TOL_FP64), ('mixed', TOL_MIXED)):
        for _ in each_candidate(h, precision):
            compare(run_gpu(h, F, q, s, S, U, precision), outs, h.nmax, tol)


@pytest.mark.parametrize('names', [['c1'], ['c2'], ['c5a', 'c5b', 'c5c']])
def test_every_tile_configuration_matches_oracle(names):
    # every compiled configuration (and the autotuner's pick) meets the
    # mixed-form gate on mid-Newton states
    import os
    if not all(os.path.exists(rom_path(nm)) for nm in names):
        pytest.skip('ROM files not generated')
    h, oroms = _handle(names)
    n = 21
    types = syn.type_labels(syn.SEED_BASE + 70, n, len(names)) if len(names) > 1 else None
    F = np.zeros((n, 2, 2))
    q = np.zeros((n, h.nmax))
    s = np.zeros((n, h.nmax))
    S = np.zeros((n, h.nmax, 3))
    U = np.zeros((n, 3))
    for t in range(len(names)):
        sel = np.arange(n) if types is None else np.nonzero(types == t)[0]
        Fm, qm, sm, Sm, Um = mid_newton_inputs(oroms[t], len(sel), syn.SEED_BASE + 71 + t)
        k = oroms[t].n
        F[sel], q[sel, :k], s[sel, :k], S[sel, :k], U[sel] = Fm, qm, sm, Sm, Um
    outs = oracle_batch(oroms, F, q, s, S, U, types)
    for precision, tol in (('fp64', TOL_FP64), ('mixed', TOL_MIXED)):
        counts = [rv.rve_rom_select_kernel(h, t, precision) for t in range(len(names))]
        for c in range(max(counts)):
            for t in range(len(names)):
                rv.rve_rom_select_kernel(h, t, precision, min(c, counts[t] - 1))
            compare(run_gpu(h, F, q, s, S, U, precision, types=types), outs, h.nmax, tol)
        ms = rv.rve_rom_autotune(h, precision, n_sample=2048)
        assert np.all(ms[:, 0] > 0)
        for t in range(len(names)):
            # the candidate in use is the fastest one, and every candidate names itself
            infos = [rv.rve_rom_kernel_info(h, t, precision, c) for c in range(counts[t])]
            assert all(nm and nl in (1, 2) for nm, nl in infos)
            assert rv.rve_rom_kernel_info(h, t, precision) == infos[int(np.argmin(ms[t, :counts[t]]))]
        compare(run_gpu(h, F, q, s, S, U, precision, types=types), outs, h.nmax, tol)


def tensor_core_candidates(h, t=0):
    """(index, name) of every tcgen05 candidate of type t (mixed form)."""
    nc = rv.rve_rom_select_kernel(h, t, 'mixed')
    names = [rv.rve_rom_kernel_info(h, t, 'mixed', c)[0] for c in range(nc)]
    return [(c, nm) for c, nm in enumerate(names) if nm.startswith('tcgen05')]


@pytest.mark.parametrize('name,kind', [('c1', 'single-role'), ('c2', 'single-role'), ('c2', 'warp-specialized'),
                                       ('c5b', 'wide'), ('c5c', 'wide')])
def test_tensor_core_kernel_many_tiles(name, kind):
    # each tcgen05 candidate, selected by name, in the launch configuration of
    # the benchmark: a persistent grid of one CTA per SM working through at
    # least 3 tiles of points each (the cross-tile phase bookkeeping of its
    # mbarriers), with a ragged last tile.  Element-wise against the SIMT
    # mixed kernel on every point, and against the oracle on 40 sampled
    # mid-Newton points at the mixed-form gate.
    import os
    import re
    if not os.path.exists(rom_path(name)):
        pytest.skip('ROM file not generated')
    h, oroms = _handle([name])
    orom = oroms[0]
    pick = {'single-role': lambda nm: 'helper' not in nm,
            'warp-specialized': lambda nm: 'helper' in nm and 'wide' not in nm,
            'wide': lambda nm: 'wide' in nm}[kind]
    cands = [(c, nm) for c, nm in tensor_core_candidates(h) if pick(nm)]
    assert len(cands) == 1, cands
    cand, cname = cands[0]
    n_pts_cta = int(re.search(r'(\d+) points', cname).group(1))
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    n = 3 * n_sm * n_pts_cta + n_pts_cta // 2 + 5       # >= 3 tiles per CTA, last tile ragged
    assert (n + n_pts_cta - 1) // n_pts_cta >= 3 * n_sm and n % n_pts_cta != 0
    idx = np.sort(syn.rng(11).choice(n, 40, replace=False))
    F = syn.fbar_batch(syn.SEED_BASE + 40, 2, n, 0.1, 0.3)
    q = np.zeros((n, h.nmax))
    s = np.zeros((n, h.nmax))
    S = np.zeros((n, h.nmax, 3))
    U = np.tile([1.0, 1.0, 0.0], (n, 1))
    # mid-Newton states everywhere: micro Newton iterations at fixed F with
    # the float64 form, then a relative perturbation of q (the mixed-form
    # error is a fraction of the Newton correction, so fresh states far from
    # equilibrium would compare the two kernels' float32 solve errors)
    rv.rve_rom_select_kernel(h, 0, 'fp64', 0)
    for _ in range(4):
        g = run_gpu(h, F, q, s, S, U, 'fp64')
        q, s, S, U = g['q'], g['s'], g['S'], g['Uprev']
    q = q + syn.perturbation(syn.SEED_BASE + 42, q.shape, 1.0) * 1e-3 * np.abs(q).max(axis=1, keepdims=True)
    # the sampled points carry states the oracle converged (inputs from the
    # oracle only, so that the comparison does not rest on the GPU)
    Fm, qm, sm, Sm, Um = mid_newton_inputs(orom, len(idx), syn.SEED_BASE + 41)
    F[idx], q[idx], s[idx], S[idx], U[idx] = Fm, qm, sm, Sm, Um
    rv.rve_rom_select_kernel(h, 0, 'mixed', 0)
    ref = run_gpu(h, F, q, s, S, U, 'mixed')
    rv.rve_rom_select_kernel(h, 0, 'mixed', cand)
    assert rv.rve_rom_kernel_info(h, 0, 'mixed')[0] == cname
    g = run_gpu(h, F, q, s, S, U, 'mixed')
    assert np.all(g['status'] == 0) and np.all(ref['status'] == 0)
    scale = np.abs(ref['Pbar']).max(axis=1)
    assert np.max(np.abs(g['Pbar'] - ref['Pbar']).max(axis=1) / scale) <= 2e-8
    tscale = np.abs(ref['dPdF']).max(axis=(1, 2))
    assert np.max(np.abs(g['dPdF'] - ref['dPdF']).max(axis=(1, 2)) / tscale) <= 2e-5
    assert np.array_equal(g['q'], ref['q']) and np.array_equal(g['Uprev'], ref['Uprev'])
    compare({k: v[idx] for k, v in g.items()}, oracle_batch(oroms, F[idx], q[idx], s[idx], S[idx], U[idx]),
            h.nmax, TOL_MIXED)
    # a second call on the same inputs: the same results (no state left
    # behind in the workspace records or the per-CTA phase counters)
    g2 = run_gpu(h, F, q, s, S, U, 'mixed')
    for k in ('Pbar', 'dPdF', 's', 'S', 'q', 'rnorm', 'status'):
        assert np.array_equal(g2[k], g[k]), k


@pytest.mark.parametrize('name,n_keep', [('c1', 10), ('c2', 20), ('c2', 17), ('c5b', 28), ('c5c', 40)])
def test_truncated_rom_every_candidate(name, n_keep):
    # a ROM with fewer modes than its tile configuration holds (padding rows
    # and columns of the augmented system, and of the tensor-core A operand
    # and B-operand image): the first n_keep modes of a stored ROM form a
    # valid ROM, evaluated by every candidate of both forms against the oracle
    import os
    if not os.path.exists(rom_path(name)):
        pytest.skip('ROM file not generated')
    full = rv.load_rom_file(rom_path(name))
    rom = dict(full, B=np.ascontiguousarray(full['B'][:, :, :n_keep]))
    h = rv.rve_rom_create(2, [rom], rom['V0'])
    orom = reduced.Rom(rom['B'], rom['w'], rom['phase'], rom['moduli'], rom['V0'])
    n = 9
    F, q, s, S, U = mid_newton_inputs(orom, n, syn.SEED_BASE + 80 + n_keep)
    outs = oracle_batch([orom], F, q, s, S, U)
    for precision, tol in (('fp64', TOL_FP64), ('mixed', TOL_MIXED)):
        for _ in each_candidate(h, precision):
            compare(run_gpu(h, F, q, s, S, U, precision), outs, h.nmax, tol)
