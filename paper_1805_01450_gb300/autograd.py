"""torch.autograd bridge: alpha(theta) as a differentiable function of the RXY angles.

Forward and backward both come from one qvx_amplitude_grad call (the adjoint of the
pairwise contractions). For real angles theta and complex outputs alpha_b, torch hands the
backward grad_b = dL/dRe(alpha_b) + i dL/dIm(alpha_b); the angle gradient is then
dL/dtheta_p = sum_b Re(conj(grad_b) * d alpha_b / d theta_p).
"""
import torch


class AmplitudeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, thetas, plan, bitstrings):
        alpha, dalpha = plan.amplitude_grad(bitstrings, thetas.detach())
        ctx.save_for_backward(dalpha)
        ctx.device = thetas.device
        return alpha

    @staticmethod
    def backward(ctx, grad_alpha):
        (dalpha,) = ctx.saved_tensors
        g = (grad_alpha.conj().unsqueeze(1) * dalpha).real.sum(0)
        return g.to(ctx.device), None, None


def amplitude(plan, bitstrings, thetas):
    """alpha_b for each bitstring, differentiable in `thetas` (float64, one per parameter)."""
    return AmplitudeFn.apply(thetas, plan, bitstrings)
