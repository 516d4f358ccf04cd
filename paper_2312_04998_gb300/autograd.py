"""torch.autograd.Function around the integrator and its discrete adjoint.

y_N = Integrate.apply(k, y0, state, t_end, C) integrates C cells with
sm_integrate; backward runs sm_adjoint with grad_output as the cotangent, so
gradients reach k (dPhi/dk_j = (dPhi/d log k_j) / k_j, 0 where k_j = 0) and y0.
The state must record steps (opts.record_steps > 0) and must not run another
integration between forward and backward: the adjoint differentiates the last
recorded run, and a stale record is refused.
"""
import torch

from . import binding as B


class Integrate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, k, y0, state, t_end, C):
        y = y0.detach().clone()
        code = state.integrate(k.detach(), y, t_end, C)
        if code != B.SM_OK:
            raise B.StoichError(code, "sm_integrate (some cells did not reach t_end)")
        ctx.state = state
        ctx.generation = state.generation
        ctx.save_for_backward(k)
        return y

    @staticmethod
    def backward(ctx, gy):
        (k,) = ctx.saved_tensors
        st = ctx.state
        if st.generation != ctx.generation:
            raise RuntimeError("the state integrated again after this forward: its record is gone")
        cot = gy.detach().contiguous().unsqueeze(0)
        grad = torch.zeros((1,) + tuple(k.shape), dtype=torch.float64, device=k.device)
        g0 = torch.zeros_like(cot) if ctx.needs_input_grad[1] else None
        code = st.adjoint(k.detach(), cot, grad, grad_y0=g0)
        if code != B.SM_OK:
            raise B.StoichError(code, "sm_adjoint")
        gk = None
        if ctx.needs_input_grad[0]:
            kd = k.detach()
            gk = torch.where(kd != 0, grad[0] / torch.where(kd != 0, kd, 1.0), torch.zeros_like(kd))
        return gk, (g0[0] if g0 is not None else None), None, None, None
