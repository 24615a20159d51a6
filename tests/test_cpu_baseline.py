"""The plain C++ float64 CPU baseline (cpu_baseline/, the host-core timing
baseline of the benchmark) against the oracle's reduced evaluation, element
by element on mid-Newton states, plus its status codes and its independence
of the thread count."""
import os

import numpy as np
import pytest

import cpu_baseline
import synthetic as syn
from conftest import rom_path
from oracle import reduced


def _mid_newton(orom, n, seed, eps, angle):
    F0 = syn.fbar_batch(seed, orom.d, n, eps, angle)
    F1 = F0 + syn.perturbation(seed + 1, F0.shape, 2e-3)
    q = np.zeros((n, orom.n))
    s = np.zeros((n, orom.n))
    S = np.zeros((n, orom.n, orom.ns))
    U = np.zeros((n, orom.ns))
    for a in range(n):
        o, _ = reduced.converge_point(orom, F0[a])
        q[a] = o['q'] + syn.perturbation(seed + 7 + a, orom.n, 1e-3 * np.abs(o['q']).max())
        s[a], S[a], U[a] = o['s'], o['S'], o['Uprev']
    return F1, q, s, S, U


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize('name,n,eps,angle', [('c1', 12, 0.1, 0.3), ('c2', 4, 0.15, 0.3), ('c3', 3, 0.2, 0.4)])
def test_cpu_baseline_matches_oracle(name, n, eps, angle):
    if not os.path.exists(rom_path(name)):
        pytest.skip('ROM file not generated')
    rom = dict(np.load(rom_path(name)))
    orom = reduced.Rom.load(rom_path(name))
    F, q, s, S, U = _mid_newton(orom, n, syn.SEED_BASE + 300, eps, angle)
    outs = [reduced.eval_point(orom, F[a], q[a], s[a], S[a], U[a]) for a in range(n)]
    g, used = cpu_baseline.eval_batch(rom, F, q.copy(), s.copy(), S.copy(), U.copy(), nthreads=2)
    assert used >= 1
    for a, o in enumerate(outs):
        assert g['status'][a] == o['status'] == 0
        assert _rel(g['Pbar'][a], o['Pbar'].ravel()) < 1e-12
        assert _rel(g['dPdF'][a], o['dPdF']) < 1e-10
        assert _rel(g['s'][a], o['s']) < 1e-9 and _rel(g['S'][a], o['S']) < 1e-9
        assert _rel(g['q'][a], o['q']) < 1e-14 and _rel(g['Uprev'][a], o['Uprev']) < 1e-13
        assert abs(g['rnorm'][a] - o['rnorm']) <= 1e-9 * o['rnorm']


def test_cpu_baseline_status_and_threads():
    rom = dict(np.load(rom_path('c1')))
    orom = reduced.Rom.load(rom_path('c1'))
    n = 40
    F = syn.fbar_batch(syn.SEED_BASE + 301, 2, n, 0.1, 0.3)
    F[3] = np.array([[-1.0, 0.0], [0.0, 1.0]])          # det F <= 0
    F[5, 0, 0] = np.nan                                 # non-finite input
    q = np.zeros((n, orom.n))
    q[7] = 50.0                                         # folds some ECM point
    s, S = np.zeros((n, orom.n)), np.zeros((n, orom.n, 3))
    U = np.tile([1.0, 1.0, 0.0], (n, 1))
    res = []
    for th in (1, 4):
        st = [x.copy() for x in (q, s, S, U)]
        g, used = cpu_baseline.eval_batch(rom, F, *st, nthreads=th)
        res.append(g)
    a, b = res
    assert list(a['status'][[3, 5, 7]]) == [1, 3, 1] and np.all(np.delete(a['status'], [3, 5, 7]) == 0)
    assert np.all(np.isnan(a['Pbar'][[3, 5, 7]]))
    assert np.array_equal(a['q'][7], q[7])              # failed points keep their state
    for k in ('Pbar', 'dPdF', 'q', 's', 'S', 'Uprev', 'status'):
        assert np.array_equal(np.nan_to_num(a[k]), np.nan_to_num(b[k])), k
