"""torch.autograd wrapper: the batched steady PSR solve as a differentiable function of
the log rate multipliers ln m_i (m_i scales the rate of progress q_i of reaction i).

Forward runs psr_batch_solve with rate_mult = exp(ln m); backward runs psr_batch_adjoint
(transposed solve with the converged Jacobian) and sums the per-reactor gradients over
the batch. Reactors that did not converge, or whose Jacobian did not factor, contribute
zero gradient. All arithmetic is in libpsr.
"""
import torch

from . import psr


class PSRSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, ln_mult, mech, Y_in, T_in, tau, P, Y0, T0, opts=None):
        opts = opts or psr.Options()
        mult = torch.exp(ln_mult.detach().to(torch.float64)).contiguous()
        out = psr.batch_solve(mech, Y_in, T_in, tau, P, Y0, T0, rate_mult=mult, opts=opts)
        ctx.mech = mech
        ctx.energy = opts.energy
        ctx.save_for_backward(Y_in, T_in, tau, P, out["Y"], out["T"], mult, out["status"])
        ctx.mark_non_differentiable(out["status"])
        return out["Y"], out["T"], out["status"]

    @staticmethod
    def backward(ctx, gY, gT, _gstatus):
        Y_in, T_in, tau, P, Y, T, mult, status = ctx.saved_tensors
        B, K = Y.shape
        g = torch.zeros((B, K + 1), dtype=torch.float64, device=Y.device)
        if gY is not None:
            g[:, :K] = gY
        if gT is not None:
            g[:, K] = gT
        grad, _, ok = psr.batch_adjoint(ctx.mech, Y_in, T_in, tau, P, Y, T, g.contiguous(),
                                        rate_mult=mult, energy=ctx.energy)
        conv = (status == psr.PSR_CONVERGED) | (status == psr.PSR_REFINE_FALLBACK)
        valid = conv & (ok == 1)
        grad = torch.where(valid[:, None], grad, torch.zeros_like(grad))
        return grad.sum(0), None, None, None, None, None, None, None, None


def psr_solve(ln_mult, mech, Y_in, T_in, tau, P, Y0, T0, opts=None):
    """(Y, T, status) of the batch; differentiable in ln_mult [I]."""
    return PSRSolve.apply(ln_mult, mech, Y_in, T_in, tau, P, Y0, T0, opts)
