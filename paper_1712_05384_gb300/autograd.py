"""torch.autograd interface: amplitudes of a parametrised circuit as a
differentiable function of its gate angles.

``amplitudes(plan, params, d_bits)`` returns a_b = <x_b|C(params)|0^n> for the
bitstrings in ``d_bits`` (complex128, on their device) where ``params`` holds
(theta_p, phi_p) of every RXY gate of the plan's circuit, flat in the order of
qgm_circuit_param_gates.  The plan must be made with ``gradients=True`` and
be bound.  Forward: the angles go into the plan's tables
(qgm_plan_set_params, no re-planning), then qgm_amplitudes.  Backward: the
library's adjoint elimination (qgm_amplitude_grad).

For a real loss L, torch hands the backward pass G_b = 2 dL/d(conj a_b) (its
convention for complex outputs) and expects dL/dp = Re sum_b conj(G_b)
da_b/dp; qgm_amplitude_grad takes g_b = dL/d(conj a_b) = G_b / 2 and returns
2 Re sum_b conj(g_b) da_b/dp, the same number.  Every step runs in the
library's kernels; this module only moves tensors.
"""
from __future__ import annotations

import torch


class AmplitudeFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, plan, d_bits):
        if not plan.gradients:
            raise ValueError("the plan was made without gradients=True")
        plan.set_params(params.detach().to("cpu", torch.float64).numpy())
        B = d_bits.numel()
        out = torch.empty(2 * B, dtype=torch.float64, device=d_bits.device)
        plan.amplitudes(d_bits, out, B=B)
        ctx.plan = plan
        ctx.save_for_backward(params, d_bits)
        return torch.view_as_complex(out.view(B, 2))

    @staticmethod
    def backward(ctx, grad_a):
        params, d_bits = ctx.saved_tensors
        plan = ctx.plan
        # the tables of these angles (a later forward may have changed them)
        plan.set_params(params.detach().to("cpu", torch.float64).numpy())
        g = torch.view_as_real((grad_a / 2).to(torch.complex128).contiguous()).reshape(-1).to(d_bits.device)
        d_grad = torch.empty(params.numel(), dtype=torch.float64, device=d_bits.device)
        plan.amplitude_grad(d_bits, g, d_grad, B=d_bits.numel())
        return d_grad.to(params.device, params.dtype).reshape(params.shape), None, None


def amplitudes(plan, params, d_bits):
    """Differentiable amplitudes (complex128, shape (B,)) -- see the module doc."""
    return AmplitudeFunction.apply(params, plan, d_bits)
