"""GPU parity of the offline stage (Sec. 3.2.1 snapshots and POD, Sec. 3.3
empirical cubature) against the oracle's offline functions, on oracle
inputs (RVE geometry, phases, seeded training paths)."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import law, rom, rve

pytestmark = pytest.mark.gpu
rv = pytest.importorskip('paper_2306_02687_gb300')
from paper_2306_02687_gb300 import offline  # noqa: E402

MOD = np.array([law.mu_kappa_from_E_nu(1.0, 0.3), law.mu_kappa_from_E_nu(10.0, 0.3)])


def _model(n, vf=0.2):
    return rve.PeriodicRVE(2, n, rve.phases_single_inclusion(2, n, vf), MOD)


def test_snapshots_and_linear_responses_match_oracle():
    n = 12
    m = _model(n)
    paths = syn.training_paths(syn.SEED_BASE + 310, 2, 5, 4, 0.12)
    X_or = rom.snapshots(m, paths)                         # [n_dof, n_snap]
    X, info = offline.rve_snapshots(n, m.phase, MOD, torch.tensor(paths, device='cuda'))
    torch.cuda.synchronize()
    inf = info.cpu().numpy()
    assert np.all(inf[:, 3] == 0), inf
    Xg = X.cpu().numpy().T
    err = np.abs(Xg - X_or).max() / np.abs(X_or).max()
    print('snapshots: max rel err %.2e, Newton %s, CG %s' % (err, inf[:, 0], inf[:, 1]))
    assert err <= 1e-8
    W_or = m.linear_responses()                            # [n_dof, 3]
    W, info = offline.rve_snapshots(n, m.phase, MOD, linear=True, cg_tol=1e-14)
    torch.cuda.synchronize()
    assert np.all(info.cpu().numpy()[:, 3] == 0)
    assert np.abs(W.cpu().numpy().T - W_or).max() <= 1e-10 * np.abs(W_or).max()
