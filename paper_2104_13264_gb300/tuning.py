"""Tuning of the proposal by gradient ascent on the mean log q of accepted samples.

The MH step keeps the chain exact whatever q is; making q larger on the states
the chain actually visits raises the acceptance.  Each tuning step
  1. re-evaluates the chains' cached log q with the current q (it changed),
  2. draws proposals (FP32 sampler) and runs the MH scan,
  3. takes the states the chains occupied during the scan as the batch, each with
     its residence time (the number of proposals it stayed for: an accepted
     proposal until the next acceptance, the state held before the scan until
     the first one), so that the batch is weighted like the chain's samples of
     pi; loss = -(residence-weighted mean of log q),
  4. backpropagates through tnmc_logq_backward on one half of the chains and
     takes a backtracking gradient-ascent step on the FP32 tensors, judged on the
     other half.
The weighted mean estimates E_pi[log q] = -KL(pi || q) - H(pi): maximising it
moves q towards pi.  (Weighting each accepted proposal once instead would favour
the states q already over-proposes.)
Tuning changes q while the chain runs (an adaptive chain): use it during burn-in
and freeze q for production sampling.
"""
import time

import torch

from . import autograd, binding


def residence_weights(acc):
    """acc: bool/uint8 [C, T] accept flags of one scan.  Returns (w_acc [C, T], w_held [C]):
    how many of the T proposals each accepted proposal, and the state held before the
    scan, stayed the chain's state (they sum to T per chain)."""
    A = acc.bool()
    C, T = A.shape
    j = torch.arange(T, device=A.device).expand(C, T)
    pos = torch.where(A, j, torch.full_like(j, T))
    after = torch.cat([pos[:, 1:], torch.full((C, 1), T, dtype=pos.dtype, device=A.device)], dim=1)
    nxt = after.flip(1).cummin(dim=1).values.flip(1)        # first acceptance after j (or T)
    w_acc = torch.where(A, nxt - j, torch.zeros_like(j))
    w_held = pos.min(dim=1).values                          # first acceptance (or T)
    return w_acc, w_held


def tune(env, steps=50, proposals=16384, chains=64, step=1e-2, seed=0, min_batch=64, max_backtrack=8, log=None):
    """Run `steps` tuning steps; returns a list of per-step records.

    Gradient ascent with backtracking.  The chains are split in two halves: the
    gradient comes from the states of the first half, and the update
    params + lr * grad is kept only if the weighted mean log q of the second
    half's states does not drop and none of them gets q = 0.  The clamped
    conditionals make the objective fall off a cliff where a weight crosses
    zero, which a fixed step can jump over; the held-out half keeps a step from
    fitting one batch's noise.  Otherwise lr is halved and the update retried.
    A kept step grows lr by 1.25.  The first lr moves the parameters by `step`
    of their norm.  With one chain both roles use the same states.
    """
    params = binding.get_params(env).clone()
    T = max(1, proposals // chains)
    B = chains * T
    chain = binding.init_chains(env, chains, seed=seed, precision="f32")
    lr = None
    hist = []
    for it in range(steps):
        torch.cuda.synchronize()
        t0 = time.time()
        binding.set_params(env, params)
        chain[1].copy_(binding.logq(env, chain[0], precision="f32")[0])      # cached log q under the new q
        held, held_lq = chain[0].clone(), chain[1].clone()
        sp, lq, E, fl = binding.sample(env, B, seed=seed + 1, sample_offset=it * B, precision="f32")
        acc = binding.mh_step(env, chains, T, (sp, lq, E), chain, seed=seed + 2, step_offset=it * T)
        w_acc, w_held = residence_weights(acc.view(chains, T))
        w_held = w_held * torch.isfinite(held_lq)                               # not a start outside q
        rate = int(torch.count_nonzero(w_acc)) / B
        rec = {"step": it, "acceptance": rate, "accepted": int(torch.count_nonzero(w_acc)), "loss": float("nan"),
               "lr": lr, "kept": False}
        half = chains // 2 if chains > 1 else chains
        parts = []
        for lo, hi in ((0, half), (half, chains) if chains > 1 else (0, chains)):
            wa = w_acc[lo:hi].flatten()
            idx = torch.nonzero(wa, as_tuple=False).flatten()
            hidx = torch.nonzero(w_held[lo:hi], as_tuple=False).flatten()
            batch = torch.cat([sp[lo * T:hi * T].index_select(0, idx), held[lo:hi].index_select(0, hidx)])
            w = torch.cat([wa.index_select(0, idx), w_held[lo:hi].index_select(0, hidx)]).to(torch.float64)
            parts.append((batch, w / w.sum().clamp_min(1), int(idx.numel())))
        (b_fit, w_fit, n_fit), (b_val, w_val, _) = parts
        if n_fit >= min_batch // 2 and w_val.sum() > 0:
            p = params.clone().requires_grad_(True)
            f = (w_fit * autograd.logq(p, env, b_fit)).sum()
            (g,) = torch.autograd.grad(f, p)
            rec["loss"] = -float(f.item())
            binding.set_params(env, params)
            fv = float((w_val * binding.logq(env, b_val, precision="f32")[0]).sum().item())
            rec["val_loss"] = -fv
            if lr is None:
                lr = step * float(params.norm()) / max(float(g.norm()), 1e-30)
            for _ in range(max_backtrack):
                cand = params + lr * g
                binding.set_params(env, cand)
                fc = float((w_val * binding.logq(env, b_val, precision="f32")[0]).sum().item())
                if fc == fc and fc > -float("inf") and fc >= fv:
                    params = cand
                    rec.update(kept=True, val_loss_after=-fc)
                    lr *= 1.25
                    break
                lr *= 0.5
            rec["lr"] = lr
        torch.cuda.synchronize()
        rec["seconds"] = time.time() - t0
        hist.append(rec)
        if log:
            log(rec)
    binding.set_params(env, params)
    return hist
