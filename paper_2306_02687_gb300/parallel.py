"""Data-parallel monolithic FE^2 iteration across ranks (one process per GPU).

The macro equilibrium of Sec. 2 (Eq. 6) is a sum over elements, and every
element's integration points carry their own RVE (Sec. 3), so the work of a
monolithic Newton iteration shards by element: a rank owns a contiguous
element range, computes Fbar at that range's points, evaluates their RVEs
(the batched hyper-ROM evaluation, no exchange) and adds the range's element
contributions to a residual and tangent of the whole mesh.  The one real
exchange is the sum of those partial systems, an all-reduce of one flat
buffer holding R and the CSR values of K together, plus a max-reduce of the
three convergence scalars.  The Newton correction then runs on every rank
from identical inputs (macro_solve is deterministic), so the nodal field
stays identical on all ranks without a broadcast.

Without an initialized process group every reduction is the identity, and
a single shard covering all elements reproduces the one-GPU iteration.
"""
import torch

from . import api


def element_range(n_elem, rank, world):
    """Contiguous, balanced element range [begin, end) of one rank: sizes
    differ by at most one, ranks in order, together all elements once."""
    if world < 1 or not 0 <= rank < world or n_elem < 0:
        raise ValueError('bad shard: rank %d of %d, %d elements' % (rank, world, n_elem))
    base, extra = divmod(n_elem, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def _group_size(group):
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return 1
    return dist.get_world_size(group)


def allreduce_system(buf, group=None):
    """Sum of the ranks' partial systems (R and Kvals packed in one
    contiguous float64 buffer), in place; one collective."""
    if _group_size(group) > 1:
        import torch.distributed as dist
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return buf


def allreduce_norms(norms, group=None):
    """Max over ranks of the convergence scalars (max |R_free|,
    max |R_prescribed|, max micro residual), in place.  The first two are
    already equal on every rank after allreduce_system; the third is local."""
    if _group_size(group) > 1:
        import torch.distributed as dist
        dist.all_reduce(norms, op=dist.ReduceOp.MAX, group=group)
    return norms


class MacroShard:
    """One rank's share of a monolithic Newton iteration on a macro mesh:
    the element range, the RVE states of its points and the whole-mesh
    system buffer.  Steps (all on the current CUDA device):
        evaluate(u)   Fbar, RVE evaluation and partial assembly of the range
        reduce()      all-reduce of the system and of the norms
        solve(u)      the Newton correction, u += du
    """

    def __init__(self, h, mesh, free_mask, rank=0, world=1, group=None, precision='mixed', types=None):
        self.h, self.m, self.group, self.precision = h, mesh, group, precision
        self.e_begin, self.e_end = element_range(mesh.n_elem, rank, world)
        self.ngp = mesh.n_ip // mesh.n_elem
        self.n = (self.e_end - self.e_begin) * self.ngp
        dev = torch.device('cuda')
        self.types = None
        if types is not None:
            t = torch.as_tensor(types, dtype=torch.int32).reshape(-1)
            if t.numel() != mesh.n_ip:
                raise ValueError('types must hold one label per integration point of the mesh')
            self.types = t[self.e_begin * self.ngp:self.e_end * self.ngp].contiguous().to(dev)
        self.free = torch.as_tensor(free_mask, dtype=torch.uint8).reshape(-1).to(dev)
        if self.free.numel() != mesh.n_dof:
            raise ValueError('free_mask must hold one flag per DOF')
        # R and Kvals in one buffer: one all-reduce per iteration
        self.system = torch.zeros(mesh.n_dof + mesh.nnz, dtype=torch.float64, device=dev)
        self.R = self.system[:mesh.n_dof]
        self.Kvals = self.system[mesh.n_dof:]
        self.Fbar = torch.empty(self.n, mesh.g, dtype=torch.float64, device=dev)
        self.q, self.s, self.S, self.Uprev = h.zero_state(self.n)
        self.Pbar, self.dPdF, self.rnorm, self.status = h.outputs(self.n)
        self.norms = torch.zeros(3, dtype=torch.float64, device=dev)

    def evaluate(self, u, stream=None):
        self.system.zero_()
        if self.n == 0:
            self.rnorm.zero_()
            return
        api.macro_gradient_range(self.m, self.e_begin, self.e_end, u, self.Fbar, stream)
        api.rve_rom_eval_batch(self.h, self.Fbar, self.q, self.s, self.S, self.Uprev, self.Pbar, self.dPdF,
                               self.rnorm, self.status, type=self.types, precision=self.precision, stream=stream)
        api.macro_assemble_range(self.m, self.e_begin, self.e_end, self.Pbar, self.dPdF, self.R, self.Kvals,
                                 stream)

    def reduce(self, stream=None):
        allreduce_system(self.system, self.group)
        api.macro_residual_norms(self.m, self.R, self.free, self.rnorm, self.norms, stream)
        return allreduce_norms(self.norms, self.group)

    def solve(self, u, tol=1e-12, max_iter=20000, stream=None):
        return api.macro_solve(self.m, self.Kvals, self.R, self.free, u=u, tol=tol, max_iter=max_iter,
                               stream=stream)
