"""torch.autograd wrapper of mfipm_solve / mfipm_backward."""
import torch

from . import Dense, backward, solve


class MfipmFunction(torch.autograd.Function):
    """x* = argmin tau||x||_1 + 1/2||Ax - b||^2 with a hand-written backward (the adjoint KKT
    solve of mfipm_backward at the final iterate)."""

    @staticmethod
    def forward(ctx, b, tau, A, op, params):
        if A is not None and A is not op.A:
            op = Dense(A.detach(), op.a_scale)
        x, info, zs = solve(op, b.detach(), float(tau), params, return_zs=True)
        ctx.save_for_backward(b.detach(), x, zs)
        ctx.op, ctx.params, ctx.tau = op, params, float(tau)
        ctx.tau_meta = (tau.dtype, tau.device)
        ctx.want_A = A is not None and ctx.needs_input_grad[2]
        ctx.info = info
        return x

    @staticmethod
    def backward(ctx, gx):
        b, x, zs = ctx.saved_tensors
        gbs, gts, gAs, _ = backward([ctx.op], [b], [ctx.tau], [x], [zs], [gx.contiguous()], ctx.params,
                                    want_A=ctx.want_A)
        gtau = torch.tensor(gts[0], dtype=ctx.tau_meta[0], device=ctx.tau_meta[1])
        gb = gbs[0].to(b.dtype) if ctx.needs_input_grad[0] else None
        return gb, gtau if ctx.needs_input_grad[1] else None, gAs[0] if ctx.want_A else None, None, None
