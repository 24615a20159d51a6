"""Element-sharded monolithic iteration on one GPU: the range entry points
(macro_gradient_range, macro_assemble_range) against the whole-mesh ones,
and a Newton loop whose ranks are emulated in turn on one device (their
partial systems summed in between, as the all-reduce would) against the
float64 oracle driver.  No kernel waits on another: the shards run one
after the other."""
import numpy as np
import pytest
import torch

import synthetic as syn
from synthetic import meshes
from conftest import rom_path
from oracle import reduced, macro

pytestmark = pytest.mark.gpu
rv = pytest.importorskip('paper_2306_02687_gb300')
from paper_2306_02687_gb300 import parallel  # noqa: E402


def T(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device='cuda')


@pytest.mark.parametrize('kind', ['plate', 'box'])
def test_ranges_reproduce_the_whole_mesh(kind):
    if kind == 'plate':
        X, conn = meshes.plate_with_hole(12, 10)
    else:
        X, conn = meshes.box(5, 4, 3, 1.0, 1.0, 0.5)
    d = X.shape[1]
    m = rv.macro_mesh_create(X, conn)
    g, ngp = d * d, m.n_ip // m.n_elem
    u = T(syn.perturbation(syn.SEED_BASE + 72, X.shape, 0.02))
    F = torch.empty(m.n_ip, g, dtype=torch.float64, device='cuda')
    rv.macro_gradient(m, u, F)
    P = T(syn.perturbation(syn.SEED_BASE + 73, (m.n_ip, g), 0.1))
    C = T(syn.perturbation(syn.SEED_BASE + 74, (m.n_ip, g, g), 1.0))
    R = torch.empty(m.n_dof, dtype=torch.float64, device='cuda')
    Kv = torch.empty(m.nnz, dtype=torch.float64, device='cuda')
    rv.macro_assemble(m, P, C, R, Kv)
    for world in (1, 3, 7):
        Rs = torch.zeros_like(R)
        Ks = torch.zeros_like(Kv)
        for r in range(world):
            e0, e1 = parallel.element_range(m.n_elem, r, world)
            p0, p1 = e0 * ngp, e1 * ngp
            Fr = torch.empty(p1 - p0, g, dtype=torch.float64, device='cuda')
            rv.macro_gradient_range(m, e0, e1, u, Fr)
            assert torch.equal(Fr, F[p0:p1])                       # same arithmetic per point
            rv.macro_assemble_range(m, e0, e1, P[p0:p1].contiguous(), C[p0:p1].contiguous(), Rs, Ks)
        # the same sums in another order of the atomics
        assert (Rs - R).abs().max().item() <= 1e-14 * R.abs().max().item()
        assert (Ks - Kv).abs().max().item() <= 1e-14 * Kv.abs().max().item()
    # residual only, and an empty range, add nothing else
    R2 = torch.zeros_like(R)
    rv.macro_assemble_range(m, 0, m.n_elem, P, None, R2)
    rv.macro_assemble_range(m, 3, 3, P[:0], None, R2)
    assert (R2 - R).abs().max().item() <= 1e-14 * R.abs().max().item()
    # ranges outside the mesh are refused before any launch
    for e0, e1 in ((-1, 2), (3, 2), (0, m.n_elem + 1)):
        with pytest.raises((RuntimeError, ValueError)):
            rv.macro_assemble_range(m, e0, e1, P[:max(e1 - e0, 0) * ngp].contiguous(), None, R2)


def _reduce(shards):
    """What allreduce_system and allreduce_norms do across ranks, for
    shards that live on one device."""
    tot = shards[0].system.clone()
    for s in shards[1:]:
        tot += s.system
    for s in shards:
        s.system.copy_(tot)
        rv.macro_residual_norms(s.m, s.R, s.free, s.rnorm, s.norms)
    nm = torch.stack([s.norms for s in shards]).max(0).values
    for s in shards:
        s.norms.copy_(nm)
    return nm


@pytest.mark.parametrize('world', [1, 3])
def test_sharded_newton_matches_the_oracle(world):
    """Uniaxial tension of a 4x4 Q4 square with the 16x16 / 12-mode / 60-point
    ROM to 10% in 10 load steps, the 16 elements split over `world` emulated
    ranks (6 + 5 + 5 for three): reactions and displacements match the
    oracle driver and every rank keeps the identical nodal field."""
    roms = [rv.load_rom_file(rom_path('c1'))]
    h = rv.rve_rom_create(2, roms, roms[0]['V0'])
    orom = reduced.Rom.load(rom_path('c1'))
    X, conn = meshes.rect(4, 4)
    m = rv.macro_mesh_create(X, conn)
    om = macro.MacroMesh(X, conn)
    prob = macro.uniaxial_problem(om, 0.1)
    n_steps = 10
    ref = macro.driver(prob, [orom], np.zeros(om.n_ip, dtype=np.int64), n_steps)
    free = np.ones(m.n_dof, dtype=np.uint8)
    free[prob.presc_dofs] = 0
    shards = [parallel.MacroShard(h, m, free, r, world) for r in range(world)]
    assert sum(s.n for s in shards) == m.n_ip
    us = [torch.zeros(m.n_nodes, 2, dtype=torch.float64, device='cuda') for _ in range(world)]
    pidx = T(prob.presc_dofs, torch.int64)
    pval = T(prob.presc_vals)
    react = T(prob.react_dofs, torch.int64)
    mu_m = orom.moduli[0, 0]
    reactions, iters = [], []
    for step in range(1, n_steps + 1):
        for u in us:
            u.view(-1)[pidx] = step / n_steps * pval
        for it in range(31):
            for s, u in zip(shards, us):
                s.evaluate(u)
            nr = _reduce(shards).cpu().numpy()
            if nr[0] <= 1e-10 * max(1.0, nr[1]) and nr[2] <= 1e-10 * mu_m * orom.V0:
                break
            assert it < 30
            for s, u in zip(shards, us):
                _, info = s.solve(u, tol=1e-13)
                assert info.cpu().numpy()[2] == 0
        for s in shards:
            assert s.status.numel() == 0 or s.status.max().item() == 0
        for u in us[1:]:
            assert torch.equal(u, us[0])                            # deterministic solve, no broadcast
        reactions.append(shards[0].R[react].sum().item())
        iters.append(it)
    print('world', world, 'Newton iterations', iters)
    assert max(iters) <= 6
    assert np.abs(np.array(reactions) - ref['reactions']).max() <= 1e-9 * np.abs(ref['reactions']).max()
    assert np.abs(us[0].cpu().numpy() - ref['u']).max() <= 1e-9


def test_empty_shard():
    """More ranks than elements: the surplus ranks own no element, add
    nothing and report a zero micro residual."""
    roms = [rv.load_rom_file(rom_path('c1'))]
    h = rv.rve_rom_create(2, roms, roms[0]['V0'])
    X, conn = meshes.rect(2, 1)
    m = rv.macro_mesh_create(X, conn)
    free = np.ones(m.n_dof, dtype=np.uint8)
    s = parallel.MacroShard(h, m, free, 2, 3)
    assert s.n == 0 and s.e_begin == s.e_end == 2
    u = T(syn.perturbation(syn.SEED_BASE + 75, X.shape, 0.01))
    s.evaluate(u)
    nm = s.reduce().cpu().numpy()
    assert torch.count_nonzero(s.system).item() == 0 and list(nm) == [0.0, 0.0, 0.0]
