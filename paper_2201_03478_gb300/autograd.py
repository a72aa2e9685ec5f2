"""torch.autograd wrapper of the sidelobe convolution (Sect. 2.1): gradients of
a loss of the TOD with respect to the sky a_lm and the beam b_lk.

Forward: synth_spin_maps then interp_tod.  Backward: adjoint_tod applied to
the incoming TOD gradient (the transposed interpolation, ring DFT and spin
Legendre step, then the sky x beam products).  The operator is linear in
A_{k,lm} = sum_X s^X_lm conj(b^X_lk), so backward needs only the inputs: the
cube is not kept (it is rebuilt on demand by a later forward instead of being
stored).

PyTorch's gradient of a real loss with respect to a complex tensor z is
dL/dRe z + i dL/dIm z; adjoint_tod returns exactly that packing.  Entries that
are not parameters (Im of m = 0 and k = 0 entries, beam entries with l < k) are
ignored by the forward and get zero gradient.
"""
from __future__ import annotations

import torch

from .binding import Plan, adjoint_tod, interp_tod, synth_spin_maps


class SidelobeConvolution(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sky, beam, theta, phi, psi, plan: Plan):
        maps = synth_spin_maps(plan, sky.detach(), beam.detach())
        tod = interp_tod(plan, maps, theta, phi, psi)
        del maps
        ctx.plan = plan
        ctx.save_for_backward(sky, beam, theta, phi, psi)
        return tod

    @staticmethod
    def backward(ctx, grad_tod):
        sky, beam, theta, phi, psi = ctx.saved_tensors
        want_s, want_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (want_s or want_b):
            return None, None, None, None, None, None
        gs, gb = adjoint_tod(ctx.plan, theta, phi, psi, grad_tod.detach().to(torch.float64).contiguous(),
                             sky.detach(), beam.detach(), want_sky=want_s, want_beam=want_b)
        return (gs if want_s else None), (gb if want_b else None), None, None, None, None


def sidelobe_tod(plan: Plan, sky, beam, theta, phi, psi):
    """Differentiable TOD c(theta, phi, psi) for the sky and beam (complex128
    tensors in the library's packing, on the plan's device)."""
    return SidelobeConvolution.apply(sky, beam, theta, phi, psi, plan)
