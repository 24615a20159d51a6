"""A monolithic Newton iteration (macro gradient, batched RVE evaluation,
assembly, convergence norms) captured once in a CUDA graph and replayed
gives the same results as eager launches."""
import pytest
import torch

import synthetic as syn
from synthetic import meshes
from conftest import rom_path

pytestmark = pytest.mark.gpu
rv = pytest.importorskip('paper_2306_02687_gb300')


@pytest.mark.parametrize('names', [['c1'], ['c5a', 'c5b', 'c5c']])
def test_graph_replay_matches_eager(names):
    import os
    if not all(os.path.exists(rom_path(nm)) for nm in names):
        pytest.skip('ROM files not generated')
    roms = [rv.load_rom_file(rom_path(nm)) for nm in names]
    h = rv.rve_rom_create(2, roms, roms[0]['V0'])
    X, conn = meshes.rect(8, 8)
    m = rv.macro_mesh_create(X, conn)
    n = m.n_ip
    dev = 'cuda'
    types = None
    if len(names) > 1:
        types = torch.tensor(syn.type_labels(3, n, len(names)), device=dev)
    u = torch.tensor(0.05 * X + syn.perturbation(4, X.shape, 0.003), device=dev)
    Fbar = torch.empty(n, 4, dtype=torch.float64, device=dev)
    P, C, rn, st = h.outputs(n)
    R = torch.empty(m.n_dof, dtype=torch.float64, device=dev)
    Kv = torch.empty(m.nnz, dtype=torch.float64, device=dev)
    free = torch.ones(m.n_dof, dtype=torch.uint8, device=dev)
    norms = torch.empty(3, dtype=torch.float64, device=dev)
    q, s, S, U = h.zero_state(n)

    def step():
        rv.macro_gradient(m, u, Fbar)
        rv.rve_rom_eval_batch(h, Fbar, q, s, S, U, P, C, rn, st, type=types, precision='mixed')
        rv.macro_assemble(m, P, C, R, Kv)
        rv.macro_residual_norms(m, R, free, rn, norms)

    init = [x.clone() for x in (q, s, S, U)]
    step()                      # warm-up: kernel attributes, point-list buffers
    eager = []
    for x, y in zip((q, s, S, U), init):
        x.copy_(y)
    for _ in range(3):
        step()
        eager.append([t.clone() for t in (P, C, q, R, norms)])
    for x, y in zip((q, s, S, U), init):
        x.copy_(y)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g):
            step()
    for x, y in zip((q, s, S, U), init):
        x.copy_(y)
    torch.cuda.synchronize()
    for it in range(3):
        g.replay()
        torch.cuda.synchronize()
        Pe, Ce, qe, Re, ne = eager[it]
        assert torch.equal(P, Pe) and torch.equal(C, Ce) and torch.equal(q, qe)
        assert (R - Re).abs().max().item() <= 1e-13 * Re.abs().max().item()   # atomics order
        assert st.max().item() == 0
