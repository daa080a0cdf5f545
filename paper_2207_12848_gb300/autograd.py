"""Differentiable transport solve: torch.autograd.Function over the C ABI.

Forward runs ``sweep_solve_dev`` (the batched sweep of every direction, Sec. 2.3) and backward runs
``sweep_adjoint_dev``: the transposed sweep in reversed level order, whose solution gives the
gradients of a loss L(J, Gamma) with respect to the absorption coefficient and the emissivity of
every cell (the adjoint covers problems without scattering and without periodic faces). Both
directions run in the CUDA library; this module only passes device pointers.
"""
from __future__ import annotations

import torch

from ._lib import Context, default_opts, sweep_opts


def _ready(sweep: Context):
    # The library works on the context's own stream; tensors produced on torch's current stream must
    # be complete before it reads them.
    cur = torch.cuda.current_stream(sweep.device)
    if cur.cuda_stream != sweep.stream:
        cur.synchronize()


class TransportSolve(torch.autograd.Function):
    """(kappa_abs, emissivity) -> (J, Gamma) on the mesh and directions already set on a Context.

    kappa_abs and emissivity are CUDA float64 tensors [n_cells, G]; J is the mean intensity and
    Gamma the absorbed rate, same shape and dtype. The Context's material is replaced by the inputs.
    """

    @staticmethod
    def forward(fctx, sweep: Context, kappa_abs: torch.Tensor, emissivity: torch.Tensor, opts: sweep_opts):
        ka = kappa_abs.detach().to(torch.float64).contiguous()
        em = emissivity.detach().to(torch.float64).contiguous()
        _ready(sweep)
        sweep.set_material(ka, em)
        J = torch.empty_like(ka)
        Gamma = torch.empty_like(ka)
        sweep.solve_dev(J, Gamma, opts)  # returns after the results are on the device
        fctx.sweep, fctx.opts = sweep, opts
        fctx.save_for_backward(ka, em)
        return J, Gamma

    @staticmethod
    def backward(fctx, dJ, dGamma):
        ka, em = fctx.saved_tensors
        sweep: Context = fctx.sweep
        dj = None if dJ is None else dJ.to(torch.float64).contiguous()
        dg = None if dGamma is None else dGamma.to(torch.float64).contiguous()
        _ready(sweep)
        sweep.set_material(ka, em)  # the context may have been re-used since the forward solve
        gk = torch.zeros_like(ka)
        ge = torch.zeros_like(ka)
        sweep.adjoint_dev(gk, ge, dj, dg, fctx.opts)
        return None, gk, ge, None


def transport_solve(sweep: Context, kappa_abs: torch.Tensor, emissivity: torch.Tensor,
                    opts: sweep_opts | None = None, **kw):
    """Mean intensity J and absorbed rate Gamma [n_cells, G], differentiable in kappa_abs and emissivity."""
    return TransportSolve.apply(sweep, kappa_abs, emissivity, opts or default_opts(**kw))
