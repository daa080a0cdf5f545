"""Differentiable transport solve: torch.autograd.Function over the C ABI.

Forward runs ``sweep_solve_dev`` (the batched sweep of every direction, Sec. 2.3) and backward runs
``sweep_adjoint_dev``: the transposed sweep in reversed level order, whose solution gives the
gradients of a loss L(J, Gamma) with respect to the absorption coefficient, the emissivity and, with
isotropic scattering, the scattering coefficient of every cell. With scattering the forward solve
is the source iteration of Alg. 1, with periodic faces the periodic iteration of Sec. 2.7 (or both),
and the backward pass is the transpose of that coupled system. Both directions run in the CUDA
library; this module only passes device pointers.
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
    """(kappa_abs, emissivity[, kappa_scat]) -> (J, Gamma) on the mesh and directions already set on a
    Context.

    kappa_abs, emissivity and kappa_scat (or None: no scattering) are CUDA float64 tensors
    [n_cells, G]; J is the mean intensity and Gamma the absorbed rate, same shape and dtype. The
    Context's material is replaced by the inputs.
    """

    @staticmethod
    def forward(fctx, sweep: Context, kappa_abs: torch.Tensor, emissivity: torch.Tensor, kappa_scat, opts: sweep_opts):
        ka = kappa_abs.detach().to(torch.float64).contiguous()
        em = emissivity.detach().to(torch.float64).contiguous()
        ks = None if kappa_scat is None else kappa_scat.detach().to(torch.float64).contiguous()
        _ready(sweep)
        sweep.set_material(ka, em, kappa_scat=ks)
        J = torch.empty_like(ka)
        Gamma = torch.empty_like(ka)
        sweep.solve_dev(J, Gamma, opts)  # returns after the results are on the device
        fctx.sweep, fctx.opts, fctx.has_ks = sweep, opts, ks is not None
        fctx.save_for_backward(ka, em, ks if ks is not None else torch.empty(0, dtype=torch.float64))
        return J, Gamma

    @staticmethod
    def backward(fctx, dJ, dGamma):
        ka, em, ks = fctx.saved_tensors
        ks = ks if fctx.has_ks else None
        sweep: Context = fctx.sweep
        dj = None if dJ is None else dJ.to(torch.float64).contiguous()
        dg = None if dGamma is None else dGamma.to(torch.float64).contiguous()
        _ready(sweep)
        sweep.set_material(ka, em, kappa_scat=ks)  # the context may have been re-used since the forward solve
        gk = torch.zeros_like(ka)
        ge = torch.zeros_like(ka)
        gs = torch.zeros_like(ka) if ks is not None else None
        sweep.adjoint_dev(gk, ge, dj, dg, fctx.opts, grad_kappa_scat_out=gs)
        return None, gk, ge, gs, None


def transport_solve(sweep: Context, kappa_abs: torch.Tensor, emissivity: torch.Tensor, kappa_scat=None,
                    opts: sweep_opts | None = None, **kw):
    """Mean intensity J and absorbed rate Gamma [n_cells, G], differentiable in kappa_abs, emissivity and
    (when given) kappa_scat."""
    return TransportSolve.apply(sweep, kappa_abs, emissivity, kappa_scat, opts or default_opts(**kw))
