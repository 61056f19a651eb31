"""Tuning of the proposal by gradient ascent on the mean log q of accepted samples.

The MH step keeps the chain exact whatever q is; making q larger on the states
the chain actually visits raises the acceptance.  Each tuning step
  1. re-evaluates the chains' cached log q with the current q (it changed),
  2. draws proposals (FP32 sampler) and runs the MH scan,
  3. takes the accepted proposals as the batch, loss = -mean log q over them,
  4. backpropagates through tnmc_logq_backward and updates the FP32 tensors.
Tuning changes q while the chain runs (an adaptive chain): use it during burn-in
and freeze q for production sampling.
"""
import time

import torch

from . import autograd, binding


def tune(env, steps=50, proposals=16384, chains=64, lr=1e-3, seed=0, min_batch=64, log=None):
    """Run `steps` tuning steps; returns a list of per-step records."""
    params = binding.get_params(env).clone().requires_grad_(True)
    opt = torch.optim.Adam([params], lr=lr)
    T = max(1, proposals // chains)
    B = chains * T
    chain = binding.init_chains(env, chains, seed=seed, precision="f32")
    hist = []
    for it in range(steps):
        torch.cuda.synchronize()
        t0 = time.time()
        binding.set_params(env, params.detach())
        chain[1].copy_(binding.logq(env, chain[0], precision="f32")[0])      # cached log q under the new q
        sp, lq, E, fl = binding.sample(env, B, seed=seed + 1, sample_offset=it * B, precision="f32")
        acc = binding.mh_step(env, chains, T, (sp, lq, E), chain, seed=seed + 2, step_offset=it * T)
        idx = torch.nonzero(acc, as_tuple=False).flatten()
        rate = idx.numel() / B
        loss_v = float("nan")
        if idx.numel() >= min_batch:
            batch = sp.index_select(0, idx)
            loss = -autograd.logq(params, env, batch).mean()
            opt.zero_grad()
            loss.backward()
            opt.step()
            loss_v = float(loss.item())
        torch.cuda.synchronize()
        rec = {"step": it, "acceptance": rate, "accepted": int(idx.numel()), "loss": loss_v,
               "seconds": time.time() - t0}
        hist.append(rec)
        if log:
            log(rec)
    binding.set_params(env, params.detach())
    return hist
