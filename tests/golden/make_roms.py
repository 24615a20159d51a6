"""Write the hyper-ROM files consumed by both the CUDA path and the oracle.

Calls only the CPU oracle (oracle/) and the seeded generators (synthetic/).
Usage:  python tests/golden/make_roms.py c1 c2 ...

Each file holds, per RVE type, the gradient table B [m~, g, n~] of the POD
modes at the ECM points, the ECM weights w [m~], the phase of each ECM point
and the moduli (mu, kappa) of the two phases (matrix E = 1, nu = 0.3;
inclusion E = 10, nu = 0.3), plus provenance metadata.

Workloads (synthetic stand-ins for the paper's RVEs, which are not public):
  c1  2D, 16x16 Q4, one centred circular inclusion (vf 0.2), 20 training
      paths x 10 steps with ||eps||_F <= 0.10, 12 modes, 60 ECM points
  c2  2D, 48x48 Q4, 4 seeded non-overlapping circles (vf 0.3), 20 x 10
      paths with ||eps||_F <= 0.15, 24 modes, 200 ECM points
  c3  3D, 16^3 hex8, centred sphere (vf 0.25), 10 x 5 paths with
      ||eps||_F <= 0.20, 40 modes, 400 ECM points
  c5a/b/c  2D, 32x32 Q4 with 1 / 3 / 6 seeded circles (vf 0.3), 20 x 10
      paths with ||eps||_F <= 0.14, 16 / 32 / 64 modes, 120 / 300 / 600
      ECM points (the three RVE types of the mixed batch)
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synthetic as syn                      # noqa: E402
from oracle import law, rom, rve            # noqa: E402

CONFIGS = {
    'c1': dict(d=2, n=16, incl=1, vf=0.20, paths=20, steps=10, eps=0.10, modes=12, ecm=60, seed=1),
    'c2': dict(d=2, n=48, incl=4, vf=0.30, paths=20, steps=10, eps=0.15, modes=24, ecm=200, seed=2),
    'c3': dict(d=3, n=16, incl=1, vf=0.25, paths=10, steps=5, eps=0.20, modes=40, ecm=400, seed=3),
    'c5a': dict(d=2, n=32, incl=1, vf=0.30, paths=20, steps=10, eps=0.14, modes=16, ecm=120, seed=51, random=True),
    'c5b': dict(d=2, n=32, incl=3, vf=0.30, paths=20, steps=10, eps=0.14, modes=32, ecm=300, seed=53),
    'c5c': dict(d=2, n=32, incl=6, vf=0.30, paths=20, steps=10, eps=0.14, modes=64, ecm=600, seed=56),
}


def moduli():
    mu_m, ka_m = law.mu_kappa_from_E_nu(1.0, 0.3)
    mu_i, ka_i = law.mu_kappa_from_E_nu(10.0, 0.3)
    return np.array([[mu_m, ka_m], [mu_i, ka_i]])


def build_rve(c):
    d, n = c['d'], c['n']
    if c['incl'] == 1 and not c.get('random', False):
        ph = rve.phases_single_inclusion(d, n, c['vf'])
    else:
        if d == 2:
            r = (c['vf'] / (c['incl'] * np.pi)) ** 0.5
        else:
            r = (3.0 * c['vf'] / (4.0 * np.pi * c['incl'])) ** (1.0 / 3.0)
        centres = syn.inclusion_centres(syn.SEED_BASE + 1000 + c['seed'], d, c['incl'], r, 1.0 / n)
        ph = rve.phases_random_inclusions(d, n, centres, r)
    return rve.PeriodicRVE(d, n, ph, moduli())


def make(name):
    c = CONFIGS[name]
    t0 = time.time()
    model = build_rve(c)
    paths = syn.training_paths(syn.SEED_BASE + c['seed'], c['d'], c['paths'], c['steps'], c['eps'])
    X = rom.snapshots(model, paths)
    Phi = rom.pod_basis(model, X, c['modes'])
    fk = rom.ecm_training(model, Phi, paths)
    xf = rom.training_matrix(fk, model.ip_weight, model.V0, c['modes'])
    del fk
    z, w = rom.ecm(xf, model.V0, c['ecm'])
    hr = rom.hyper_rom(model, Phi, z, w)
    out = os.path.join(HERE, 'rom_%s.npz' % name)
    rom.save_rom(out, hr, ecm_index=z, vf=model.phase.mean(), mesh_n=c['n'],
                 n_training=X.shape[1])
    print('%s: d=%d n_dof=%d modes=%d ecm=%d sum(w)=%.15f min(w)=%.3e vf=%.4f  %.1fs'
          % (name, c['d'], model.n_dof, hr.n, hr.m, w.sum(), w.min(), model.phase.mean(),
             time.time() - t0))


if __name__ == '__main__':
    for name in sys.argv[1:]:
        make(name)
