"""torch.autograd.Function around the inverse NFFT (the differentiable form).

forward : fhat = D^* F^* B_opt(x)^* f   (set_nodes + precompute + infft_apply on a plan of
          its own, kept for the backward)
backward: grad_f = B_opt F D w (nfft_apply, the exact adjoint)
          grad_x = infft_grad_nodes (implicit differentiation of the column problems)
where w is the incoming gradient with respect to fhat.  Every step runs in the CUDA
library; this module only wires the calls."""
import torch

from . import binding as _b


class InverseNFFT(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, x, M, sigma, m, tau):
        if not (f.is_cuda and x.is_cuda):
            raise ValueError("inverse_nfft needs CUDA tensors")
        f = f.contiguous().to(torch.complex64)
        x = x.contiguous().to(torch.float64)
        plan = _b.infft_plan_create(M, x.shape[0], sigma, m, tau=tau)
        _b.infft_set_nodes(plan, x)
        _b.infft_precompute(plan)
        fhat = _b.infft_apply(plan, f)
        ctx.plan = plan
        ctx.save_for_backward(f)
        return fhat

    @staticmethod
    def backward(ctx, grad_fhat):
        (f,) = ctx.saved_tensors
        w = grad_fhat.contiguous().to(torch.complex64)
        grad_f = _b.nfft_apply(ctx.plan, w) if ctx.needs_input_grad[0] else None
        grad_x = _b.infft_grad_nodes(ctx.plan, f, w) if ctx.needs_input_grad[1] else None
        return grad_f, grad_x, None, None, None, None


def inverse_nfft(f, x, M, sigma=2.0, m=4, tau=1e-12):
    """Differentiable inverse NFFT: fhat (complex64, M) from samples f (N) at nodes x (N, float64)."""
    return InverseNFFT.apply(f, x, M, sigma, m, tau)
