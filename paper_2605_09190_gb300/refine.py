"""Refinement of the MP coefficients on a fixed support (differentiable
synthesis + SSIM).

The support -- leaves and atom indices of an encode -- is held fixed and the
coefficients are refined by gradient ascent on the mean SSIM (Section 3) of
the synthesised planes (Algorithm 3).  Forward and backward both run in the
library's kernels (`aqmp_synth_forward` / `aqmp_synth_backward` /
`aqmp_ssim`); this module only wraps them as a torch.autograd.Function.  The
loss uses the unclipped reconstruction (the clip of the reported metric has
no useful gradient where it saturates).
"""
from __future__ import annotations

import torch

from . import aqmp


class SynthesisSSIM(torch.autograd.Function):
    """mean over planes of SSIM(ref_p, synthesis_p(alpha)); alpha is the
    code's coefficient vector in canonical order (float32, CUDA)."""

    @staticmethod
    def forward(ctx, alpha, code, refs):
        # When alpha needs a gradient, the SSIM kernels return d SSIM / d y
        # in the same pass (the window statistics are computed once); the
        # backward only scales it and runs the synthesis adjoint.
        want = ctx.needs_input_grad[0]
        grads, vals = [], []
        for plane, ref in refs:
            out = torch.empty_like(ref)
            aqmp.aqmp_synth_forward(code, plane, alpha, out)
            s = torch.zeros((), dtype=torch.float64, device=ref.device)
            if want:
                gy = torch.empty_like(out)
                aqmp.aqmp_ssim(ref, out, s, gy, 1.0)
                grads.append(gy)
            else:
                aqmp.aqmp_ssim(ref, out, s)
            vals.append(s)
        ctx.code, ctx.refs, ctx.grads = code, refs, grads
        ctx.n_alpha = alpha.shape[0]
        return torch.stack(vals).mean()

    @staticmethod
    def backward(ctx, grad):
        grad_alpha = torch.zeros(ctx.n_alpha, dtype=torch.float32, device=grad.device)
        for (plane, _), gy in zip(ctx.refs, ctx.grads):
            aqmp.aqmp_synth_backward(ctx.code, plane, gy, grad_alpha)
        # the mean over planes and the upstream gradient, on the device
        return grad_alpha * (grad / len(ctx.refs)).to(torch.float32), None, None


def synthesis_ssim(alpha, code, refs):
    return SynthesisSSIM.apply(alpha, code, refs)


def refine(code, refs, steps: int = 50, lr: float = 0.25):
    """`steps` Adam steps of SSIM ascent from the code's own coefficients.
    `refs` is a list of (plane index, reference image as CUDA float32).
    Returns (refined alpha, SSIM history with the starting value first)."""
    _, alpha0 = aqmp.aqmp_device_atoms(code)
    alpha = alpha0.clone().requires_grad_(True)
    opt = torch.optim.Adam([alpha], lr=lr)
    history = []
    for _ in range(steps):
        opt.zero_grad(set_to_none=True)
        s = synthesis_ssim(alpha, code, refs)
        (-s).backward()
        history.append(float(s.detach()))
        opt.step()
    with torch.no_grad():
        history.append(float(synthesis_ssim(alpha, code, refs)))
    return alpha.detach(), history
