"""torch.autograd.Function over the library's hand-written adjoint.

    J = SteadyStateObjective.apply(w, alpha, spec)      # w, alpha: 0-d tensors
    J.backward()                                         # w.grad, alpha.grad

`spec` fixes everything but (w, alpha): N, Gamma, dt, seed, precision,
window_start, M, steps, checkpoint, objective ("SpSm" or "g2"). The forward
pass calls twa_grad, which runs the trajectories, the reverse sweep and returns
J with its pathwise derivatives at fixed noise; backward scales them by the
incoming gradient. No arithmetic of the method happens here.
"""
import torch

from . import twa


class SteadyStateObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, alpha, spec):
        with twa.TWA(spec["N"], float(alpha), float(w), spec["Gamma"], spec["dt"], seed=spec.get("seed", 0),
                     precision=spec.get("precision", "bf16x3"), window_start=spec.get("window_start", 0.0)) as g:
            r = g.grad(spec.get("objective", "SpSm"), spec["M"], spec["steps"], spec.get("checkpoint", 64),
                       want_alpha=True)
        ctx.save_for_backward(torch.tensor([r["dJ_dw"], r["dJ_dalpha"]], dtype=torch.float64))
        ctx.se = (r["dJ_dw_se"], r["dJ_dalpha_se"])
        return torch.tensor(r["J"], dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g[0], grad_out * g[1], None
