"""torch.autograd.Function over the library's evaluate / backward pair.

    phi, grad = laplace_fmm(x, q, handle)

evaluates the potential and its gradient at the N particles x (float64,
(N, 3), CUDA) with charges q ((N,), CUDA) through ``handle.evaluate``; the
backward pass calls ``handle.backward`` (fmm_backward), the hand-written
adjoint:  dL/dq = Psi(x) and dL/dx = dL/dphi * grad + H dL/dgrad + q grad Psi,
Psi being the potential of charges dL/dphi and dipoles dL/dgrad.  Both run in
the library's CUDA kernels; this module only marshals tensors (FP32 charges
and outputs, results cast back to the inputs' dtypes).

The adjoint reads the handle's state of the evaluation it differentiates, so
a handle must not evaluate again before that backward runs; this is checked.
For the energy E = 1/2 sum q_i phi_i, autograd gives dE/dq = phi and
dE/dx = q grad with one backward call (dL/dphi = q / 2, dL/dgrad = 0).
"""
import torch

from . import fmm as _fmm


class LaplaceFMMFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, q, handle):
        if x.dtype != torch.float64:
            raise TypeError("x must be float64 (N, 3)")
        q32 = q.detach().to(torch.float32).contiguous()
        phi, grad = handle.evaluate(q32, x=x.detach().contiguous())
        ctx.handle = handle
        ctx.evaluation = handle.evaluations
        ctx.x_dtype, ctx.q_dtype = x.dtype, q.dtype
        return phi, grad

    @staticmethod
    def backward(ctx, dphi, dgrad):
        h = ctx.handle
        if h.evaluations != ctx.evaluation:
            raise RuntimeError("the FMM handle evaluated again before this backward; "
                               "use one handle per differentiated evaluation")
        dp = dphi.to(torch.float32).contiguous() if dphi is not None else None
        dg = dgrad.to(torch.float32).contiguous() if dgrad is not None else None
        dq, dx = h.backward(dp, dg, want_dq=ctx.needs_input_grad[1], want_dx=ctx.needs_input_grad[0])
        return (dx.to(ctx.x_dtype) if dx is not None else None,
                dq.to(ctx.q_dtype) if dq is not None else None, None)


def laplace_fmm(x, q, handle):
    """(phi, grad) of charges q at positions x, differentiable in x and q."""
    return LaplaceFMMFunction.apply(x, q, handle)


def make_handle(N, P=6, theta=0.4, ncrit=64, **kw):
    """An fmm.FMM handle on the current device and stream."""
    return _fmm.FMM(N, P, theta, ncrit, **kw)
