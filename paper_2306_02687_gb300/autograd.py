"""torch.autograd wrapper: homogenized stress of the converged hyper-reduced
RVE as a differentiable function of the macro deformation gradients and of
the phase moduli.

forward : repeated rve_rom_eval_batch at fixed Fbar (the monolithic update
          then reduces to micro Newton steps) until max_alpha max|r_alpha| <= tol;
          returns Pbar [n, g]
backward: rve_rom_adjoint at the converged amplitudes (implicit function
          theorem through r(q*, U, theta) = 0): gFbar = dPdF^T gPbar and
          gTheta [n_types, 2, 2] (d/d(mu, kappa) of phase 0 and 1 per type).
"""
import torch

from . import api


class RveStress(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Fbar, moduli, h, types=None, tol=1e-12, maxit=30, precision='fp64'):
        mod = moduli.detach().to('cpu', torch.float64)
        for t in range(h.n_types):
            api.rve_rom_set_moduli(h, t, mod[t].numpy())
        Fbar = Fbar.detach().contiguous()
        n = Fbar.shape[0]
        q, s, S, U = h.zero_state(n)
        Pbar, dPdF, rnorm, status = h.outputs(n)
        for _ in range(maxit):
            api.rve_rom_eval_batch(h, Fbar, q, s, S, U, Pbar, dPdF, rnorm, status, type=types,
                                   precision=precision)
            if int(status.max().item()) != 0:
                raise RuntimeError('micro evaluation failed (status %d)' % int(status.max().item()))
            if float(rnorm.max().item()) <= tol:
                break
        ctx.h = h
        ctx.types = types
        ctx.save_for_backward(Fbar, q)
        return Pbar

    @staticmethod
    def backward(ctx, gP):
        Fbar, q = ctx.saved_tensors
        h = ctx.h
        gF = torch.empty_like(Fbar)
        gth = torch.zeros(h.n_types, 2, 2, dtype=torch.float64, device=Fbar.device)
        status = torch.empty(Fbar.shape[0], dtype=torch.int32, device=Fbar.device)
        api.rve_rom_adjoint(h, Fbar, q, gP.contiguous(), gF, gth, status, type=ctx.types)
        return gF, gth, None, None, None, None, None


def rve_stress(Fbar, moduli, h, types=None, tol=1e-12, maxit=30, precision='fp64'):
    return RveStress.apply(Fbar, moduli, h, types, tol, maxit, precision)
