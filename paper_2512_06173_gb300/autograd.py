"""Transmitted flux of a coupled run as a differentiable function of the design-box
permittivity and the molecular couplings.

`CoupledFlux.apply(eps, gamma, grid, state0, nsteps, plane, freq, ckpt_every)`
returns the net flux through flux plane `plane` at frequency index `freq`
(Sec. IV spectra) accumulated over `nsteps` steps that start from the saved grid
state `state0` (bytes from `Grid.checkpoint()`), for design-box permittivities
`eps` (sz, sy, sx) and couplings `gamma` (nmol).  The gradient comes from the
library's hand-written discrete adjoint (`ml_adjoint_run`): the reverse sweep
needs the forward run's final DFT sums, so when a gradient is wanted the forward call
runs both sweeps and keeps the gradients, and backward only scales them; when neither
input needs a gradient the forward call runs the forward steps alone.  All arithmetic
runs in the library's CUDA kernels; torch provides the tensors.
"""
from __future__ import annotations

import torch

from . import maxlink


class CoupledFlux(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps, gamma, grid, state0, nsteps, plane, freq, ckpt_every=100):
        e = eps.detach().to(torch.float64).contiguous()
        gm = gamma.detach().to(torch.float64).contiguous()
        grid.restore(state0)
        maxlink.ml_set_design_eps(grid.h, e.data_ptr(), e.is_cuda, grid.stream)
        if gm.numel():
            maxlink.ml_set_couplings(grid.h, gm.data_ptr(), gm.is_cuda, grid.stream)
        need_e, need_g = ctx.needs_input_grad[0], ctx.needs_input_grad[1] and gm.numel() > 0
        dev = torch.device("cuda", torch.cuda.current_device())
        ge = torch.zeros(e.shape, dtype=torch.float64, device=dev)
        gg = torch.zeros(max(gm.numel(), 1), dtype=torch.float64, device=dev)
        obj = maxlink.ml_adjoint_run(grid.h, nsteps, ckpt_every, plane, freq, ge.data_ptr() if need_e else 0,
                                     gg.data_ptr() if need_g else 0, True, grid.stream)
        ctx.save_for_backward(ge.to(eps.device, eps.dtype), gg[:gm.numel()].to(gamma.device, gamma.dtype))
        return torch.tensor(obj, dtype=torch.float64, device=eps.device)

    @staticmethod
    def backward(ctx, grad_out):
        ge, gg = ctx.saved_tensors
        return grad_out * ge, grad_out * gg, None, None, None, None, None, None
