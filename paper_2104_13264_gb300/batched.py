"""Batched persistent form: tile autotuner and CUDA-graph step runner.

Many independent instances (disorder realisations of uneven L and chi) are
sampled by one persistent launch of the library (``tnmc_sample_batched``) and
scanned by one batched MH launch (``tnmc_mh_batched``).  This module picks the
launch shape and captures the per-step launches in a CUDA graph:

* ``autotune`` times every candidate (tile of 64 or 128 samples per work item x
  item order "instance" or "cost"-descending) on the actual workload with CUDA
  events and caches the fastest in a JSON file keyed by the workload and the
  device;
* ``BatchRunner`` owns the plan, the proposal and chain buffers, and replays a
  captured graph of sample -> MH -> advance, so a step costs one graph launch.

The arithmetic is the library's; nothing here computes.
"""
import hashlib
import json
import os

from . import binding

CACHE_PATH = os.path.join(binding.HERE, "_build", "batch_tiles.json")
CANDIDATES = [(tile, order) for tile in (64, 128) for order in ("instance", "cost")]


def workload_key(envs, B, chains, precision):
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sig = {
        "device": props.name, "sms": props.multi_processor_count, "precision": precision, "chains": int(chains),
        "inst": [[e.Lx, e.Ly, e.chi, int(b)] for e, b in zip(envs, B)],
    }
    return hashlib.sha1(json.dumps(sig, sort_keys=True).encode()).hexdigest()


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def time_plan(plan, reps=3, warmup=1, seed=0):
    """Mean milliseconds of one tnmc_sample_batched launch of `plan`."""
    import torch
    out = plan.alloc_proposals()
    plan.set_step(seed, 0)
    for _ in range(warmup):
        plan.sample(out)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(reps):
        plan.sample(out)
    t1.record()
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / reps


def autotune(envs, B, chains=1, precision="f32", cache_path=CACHE_PATH, reps=3, refresh=False, log=None):
    """Fastest (tile, order) for this workload; times every candidate once, then caches it."""
    import numpy as np
    B = [int(b) for b in np.broadcast_to(np.asarray(B), (len(envs),))]
    key = workload_key(envs, B, chains, precision)
    cache = _load(cache_path)
    if not refresh and key in cache:
        return cache[key]
    results = []
    for tile, order in CANDIDATES:
        plan = binding.Batch(envs, B, chains=chains, precision=precision, tile=tile, order=order)
        ms = time_plan(plan, reps=reps)
        plan.free()
        results.append({"tile": tile, "order": order, "ms": ms})
        if log:
            log("autotune tile=%d order=%s: %.3f ms" % (tile, order, ms))
    best = min(results, key=lambda r: r["ms"])
    best = dict(best, candidates=results)
    cache[key] = best
    os.makedirs(os.path.dirname(cache_path), exist_ok=True)
    tmp = cache_path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, cache_path)
    return best


class BatchRunner:
    """Plan + buffers + captured graph of one MH step over every instance.

    step k: proposals of every instance (tnmc_sample_batched), the MH scan of
    every chain (tnmc_mh_batched), then k += 1 on the device.
    """

    def __init__(self, envs, B, chains=1, precision="f32", tile=None, order=None, seed=0, tune=True,
                 cache_path=CACHE_PATH, log=None, sweeps=0):
        import torch
        if tile is None or order is None:
            if tune:
                best = autotune(envs, B, chains, precision, cache_path=cache_path, log=log)
                tile, order = best["tile"], best["order"]
            else:
                tile, order = 128, "cost"
        self.plan = binding.Batch(envs, B, chains=chains, precision=precision, tile=tile, order=order)
        self.seed = seed
        self.prop = self.plan.alloc_proposals()
        self.chain = self.plan.init_chains(seed)
        inf = self.plan.info()
        self.accepted = torch.zeros(inf["proposal_rows"], dtype=torch.uint8, device="cuda")
        self.n_accepted = torch.zeros(self.plan.n, dtype=torch.int64, device="cuda")
        self.plan.set_step(seed, 0)
        self.sweeps = int(sweeps)
        self.graph = None

    def _launch(self):
        self.plan.sample(self.prop)
        self.plan.mh(self.prop, self.chain, self.accepted, self.n_accepted)
        if self.sweeps:
            # single-spin-flip Metropolis sweeps between proposals (Sec. 3, Table hb)
            self.plan.metropolis(self.chain, self.sweeps)
        self.plan.advance()

    def delta(self):
        """The equilibration diagnostic of Sec. 3 (eq. Delta) over the plan's instances:
        the mean over instances of (1/|V|)(<H> + beta (|E| - sum <s_i s_j>^2)), with <H> the
        chains' mean energy and the link overlap averaged over replica pairs (2k, 2k+1).
        It vanishes at equilibrium on average over Gaussian disorder."""
        import torch
        q = self.plan.link_overlap(self.chain[0]).mean(dim=1)
        E = self.chain[2].view(self.plan.n, self.plan.chains).mean(dim=1)
        dims = torch.tensor([[e.Lx, e.Ly, e.beta] for e in self.plan.envs], dtype=torch.float64, device=E.device)
        Lx, Ly, beta = dims[:, 0], dims[:, 1], dims[:, 2]
        nb = Ly * (Lx - 1) + (Ly - 1) * Lx
        d = (E + beta * (nb - q)) / (Lx * Ly)
        return float(d.mean().item()), d

    def step_eager(self):
        self._launch()

    def capture(self):
        """Capture one step in a CUDA graph (the launches allocate nothing)."""
        import torch
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            self._launch()
        torch.cuda.synchronize()
        self.graph = g
        return g

    def step(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()


class MixedRunner:
    """MH steps over many instances with the sampler chosen per chi class: instances with
    chi < tc_chi share one persistent FP32 plan (BatchRunner, graph replay); each instance
    with chi >= tc_chi draws its proposals with the BF16 tensor-core sampler (tnmc_sample)
    and runs its own MH scan (tnmc_mh_step), on a stream of its own, concurrently with the
    plan.  The small instances are the plan's instances 0 .. n_small - 1 with the plan's
    counters; the j-th large one has instance index n_small + j, so at step k it draws
    sample indices ((n_small + j) << 40) + k B and MH step offsets ((n_small + j) << 40) + k T
    (chain c of the instance is MH chain c): every instance has its own random streams."""

    def __init__(self, insts, B, chains, tc_chi=32, seed=0, tune=True, log=None):
        import torch
        self.B, self.C, self.T = int(B), int(chains), int(B) // int(chains)
        self.seed = int(seed)
        self.small_idx = [i for i, x in enumerate(insts) if x.chi < tc_chi]
        self.big_idx = [i for i, x in enumerate(insts) if x.chi >= tc_chi]
        self.small_envs = binding.build_envs_batched([insts[i] for i in self.small_idx], precisions=("f32",)) \
            if self.small_idx else []
        self.big_envs = binding.build_envs_batched([insts[i] for i in self.big_idx], precisions=("bf16",)) \
            if self.big_idx else []
        self.small = BatchRunner(self.small_envs, B, chains=chains, precision="f32", seed=seed, tune=tune,
                                 log=log) if self.small_envs else None
        dev = torch.device("cuda")
        # the tensor-core instances go first and on high-priority streams, largest first, so
        # that their long tiles start before the persistent plan fills the SMs
        try:
            hi = torch.cuda.Stream.priority_range()[1]
        except (AttributeError, RuntimeError):
            hi = 0
        self.streams = [torch.cuda.Stream(priority=hi) for _ in self.big_envs]
        self.order = sorted(range(len(self.big_envs)), key=lambda j: -self.big_envs[j].Lx * self.big_envs[j].Ly)
        self.big_prop, self.big_chain = [], []
        for e in self.big_envs:
            self.big_prop.append((torch.empty((self.B, e.Ly, e.Lx), dtype=torch.int8, device=dev),
                                  torch.empty(self.B, dtype=torch.float64, device=dev),
                                  torch.empty(self.B, dtype=torch.float64, device=dev),
                                  torch.empty(self.B, dtype=torch.int32, device=dev)))
            self.big_chain.append(binding.init_chains(e, self.C, seed=seed + 1, precision="bf16"))
        self.big_accepted = torch.zeros(len(self.big_envs), dtype=torch.int64, device=dev)
        self.k = 0

    def step(self):
        import torch
        cur = torch.cuda.current_stream()
        k = self.k
        for j in self.order:
            e, s = self.big_envs[j], self.streams[j]
            s.wait_stream(cur)
            i = len(self.small_idx) + j
            sp, lq, E, fl = self.big_prop[j]
            binding.sample(e, self.B, seed=self.seed, sample_offset=(i << 40) + k * self.B, precision="bf16",
                           out=(sp, lq, E, fl), stream=s)
            binding.mh_step(e, self.C, self.T, (sp, lq, E), self.big_chain[j], seed=self.seed,
                            step_offset=(i << 40) + k * self.T, n_accepted=self.big_accepted[j:j + 1], stream=s)
        if self.small is not None:
            self.small.step()
        for s in self.streams:
            cur.wait_stream(s)
        self.k += 1

    def n_accepted(self):
        tot = int(self.big_accepted.sum().item())
        if self.small is not None:
            tot += int(self.small.n_accepted.sum().item())
        return tot

    def reset_counts(self):
        self.big_accepted.zero_()
        if self.small is not None:
            self.small.n_accepted.zero_()

    def flagged_fraction(self):
        import torch
        fl = [p[3] for p in self.big_prop]
        if self.small is not None:
            fl.append(self.small.prop[3])
        return float(torch.cat([f.flatten() for f in fl]).ne(0).double().mean().item())
