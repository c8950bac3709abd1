"""torch.autograd.Function over the tracking cost of a horizon.

cost_i = sum over frames f of the horizon of
    sum_l w_force |c_il,f - o_l,f|^2 + w_contact (contact-state mismatch)
(Sec. III-C on the frame step of Sec. III-A) for every environment i of a
handle, as a differentiable function of the initial pose (position and the
quaternion's components, in the handle's [N][8] layout) and the parameters
(mass, friction). The forward sets the state through sim_set_state and calls
sim_adjoint, which returns the costs and their gradients in one pass; the
backward only scales the stored gradients by the incoming ones. All
arithmetic runs in libinhand.so.
"""
from __future__ import annotations

import torch


class TrackingCost(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pose, params, vel, sim, frame0, obs, checkpoint_every, beta, width):
        sim.sim_set_state(pose.detach().contiguous(), vel.detach().contiguous(), params.detach().contiguous())
        cost, grad, grad_q = sim.sim_adjoint(frame0, obs, checkpoint_every=checkpoint_every, beta=beta,
                                             width=width, want_quat=True)
        gp = torch.zeros_like(pose)
        gp[:, 0:3] = grad[:, 0:3]
        gp[:, 4:8] = grad_q
        ctx.save_for_backward(gp, grad[:, 6:8].contiguous())
        return cost

    @staticmethod
    def backward(ctx, g):
        gp, gparams = ctx.saved_tensors
        s = g.to(gp.dtype)[:, None]
        return gp * s, gparams * s, None, None, None, None, None, None, None


def tracking_cost(sim, pose, params, vel, frame0: int, obs, checkpoint_every: int = 10, beta: float = 1e3,
                  width: float = 1e-3):
    """Differentiable horizon cost (float64[N]) of every environment of `sim`
    from state (pose [N][8], vel [N][8], params [N][2]) at the start of frame0,
    against observations obs [H][P][3]. Gradients flow to pose (position and
    quaternion components) and params; the velocity is held fixed."""
    return TrackingCost.apply(pose, params, vel, sim, frame0, obs, checkpoint_every, beta, width)
