"""torch.autograd wrapper of the forced log q and its hand-written backward.

LogQ.apply(params, env, spins) -> log q [B] (float64) for the FP32 sampler
tensors `params` (flat, as binding.get_params returns them); backward calls
tnmc_logq_backward with the incoming gradient as the sample weights.  Samples
with log q = -inf get weight 0 (their log q has no derivative).

The env holds one set of tensors at a time.  Forward installs `params`; since
the env may have been given other tensors before backward runs (a second
LogQ in the same graph, a tuning step in between), backward installs the
forward's `params` again, so the gradient is always taken at the point the
forward evaluated.  The env is left holding those tensors.
"""
import torch

from . import binding


class LogQ(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, env, spins):
        binding.set_params(env, params)
        lq, _, _ = binding.logq(env, spins, precision="f32")
        ctx.env = env
        ctx.save_for_backward(params, spins, lq)
        return lq

    @staticmethod
    def backward(ctx, g):
        params, spins, lq = ctx.saved_tensors
        binding.set_params(ctx.env, params)
        w = torch.where(torch.isfinite(lq), g, torch.zeros_like(g)).float()
        grad = binding.logq_backward(ctx.env, spins, w)
        return grad, None, None


def logq(params, env, spins):
    return LogQ.apply(params, env, spins)
