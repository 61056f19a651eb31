"""Benchmark of the TNMH proposal path: accepted samples/s (and proposals/s).

One step = draw B proposals (tnmc_sample) + the MH scan of C chains over them
(tnmc_mh_step), on an environment built beforehand (the build is amortised
over the chain and reported separately as env_build_s).  Inputs are synthetic
instances from paper_2104_13264_gb300.instances.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config c5] [--precision bf16]
  python bench.py --impl reference ...   # the FP64 CPU oracle on a bounded sample

N > 1 (torchrun): independent replicas, rank i draws sample indices
[i B, (i+1) B); no collective on the data path; timing is the max over ranks.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CONFIGS = {
    # name: (instance factory, B, chains C, default precision, description)
    "c1": ("config1", 10000, 1, "f64", "8x8 ferromagnet, beta=0.44, chi=8, 10^4 proposals, 1 chain"),
    "c2": ("config2", 65536, 256, "f32", "32x32 +-J EA, beta=1.0, chi=16, B=65536"),
    "c3": ("config3", 4096, 16, "f32", "256 Gaussian EA instances, L in {16,24,32,48,64}, chi in {8,16,32}, "
                                       "beta=2.0, 4096 proposals each, one persistent graph-captured launch"),
    "c4": ("config4", 16384, 64, "f32", "64x64 fully frustrated, beta=1.5, chi=32, B=16384"),
    "c5": ("config5", 1 << 20, 1024, "bf16", "256x256 ferromagnet, beta=0.4407, chi=64, B=2^20"),
    "c5p": ("config5_strip", 65536, 64, "bf16", "16x256 ferromagnet strip (Lx, beta, chi of the 256x256 case), "
                                               "B=65536: profiling case of the sampler kernels"),
    "c3p": ("gaussian_ea_torus_batch", 16, 16, "f64", "32 Gaussian EA disorder samples on 32x32 tori, T=0.212, chi=16, "
                                                       "16 chains each: frozen-line TNMH moves (random cuts), Delta diagnostic"),
    "c3d": ("gaussian_ea_batch", 32, 32, "f64", "256 Gaussian EA instances 32x32, T=0.212, chi=16, 32 chains each: "
                                               "TNMH move + one Metropolis sweep per iteration, Delta diagnostic"),
    "c6": ("cubic_ferromagnet", 65536, 512, "f32", "16x16x16 ferromagnet (open boundaries), T=4.5, D=2, chi=2, bond basis: "
                                                 "3D TNMH proposals + MH (Sec. 3D, rejection-rate figure setting)"),
}

# the paper's Table hb row for TNMH + Metropolis: iterations to reach each Delta threshold
# (10^4 disorders, 30 chains; hardware unstated) -- context for the measured counts
TABLE_HB = {"thresholds": [0.25, 0.15, 0.05, 0.025], "tnmh_plus_metropolis": [3, 3, 5, 5]}
# Table hbpbc (periodic boundaries, frozen-line moves): TNMH iterations (upper bounds)
TABLE_HBPBC = {"thresholds": [0.25, 0.15, 0.05, 0.025], "tnmh": [14, 21, 40, 56]}


def algorithmic_flops(inst, gauge="spin"):
    """8 chi_c chi_{c+1} FLOP per site per sample for rows r >= 1, 4 chi chi' for row 0
    (its right sweep does not depend on the sample): the left and right sweeps.  In the
    bond gauge row r is sampled from bonds 2 chi'_c of the truncated env'_{r+1} (2 on the
    last row)."""
    Lx, Ly, chi = inst.Lx, inst.Ly, inst.chi

    def bd_env(r, c):
        if c <= 0 or c >= Lx:
            return 1
        return min(chi, 1 << min(c, Lx - c, Ly - r, 30))

    def bd(r, c):
        if gauge == "spin":
            return bd_env(r, c)
        if c <= 0 or c >= Lx:
            return 1
        return 2 * (bd_env(r + 1, c) if r + 1 < Ly else 1)

    tot = 0
    for r in range(Ly):
        for c in range(Lx):
            tot += (8 if r > 0 else 4) * bd(r, c) * bd(r, c + 1)
    return tot


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_tnmc(args):
    import torch
    from paper_2104_13264_gb300 import binding as Bd
    from paper_2104_13264_gb300 import instances, replicas

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    fac, Bdef, Cdef, pdef, desc = CONFIGS[args.config]
    inst = getattr(instances, fac)()
    B = args.batch or Bdef
    C = args.chains or Cdef
    assert B % C == 0
    T = B // C
    prec = args.precision or pdef
    dev = torch.device("cuda", local)

    t0 = time.time()
    env = Bd.Env.from_instance(inst, precisions=tuple(sorted({"f64", prec} | ({"f32"} if args.tune_steps else set()))),
                               gauge=args.gauge)
    info = env.info()
    env_build_s = time.time() - t0
    tuning = None
    if args.tune_steps:
        # gradient ascent of the FP32 tensors on the chain states' mean log q (hand-written
        # backward of log q); the timed sampling below then uses the tuned FP32 copy
        from paper_2104_13264_gb300 import tuning as tn
        assert prec == "f32", "tuning acts on the FP32 sampler copy"
        torch.cuda.synchronize()
        t1 = time.time()
        hist = tn.tune(env, steps=args.tune_steps, proposals=B, chains=C, seed=args.seed + 11)
        torch.cuda.synchronize()
        tune_s = time.time() - t1
        # backward-kernel time on one batch of B proposals (CUDA events on its stream)
        sp_b = Bd.sample(env, B, seed=args.seed + 13, precision="f32")[0]
        wts = torch.full((B,), 1.0 / B, dtype=torch.float32, device=dev)
        Bd.logq_backward(env, sp_b, wts)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record()
        Bd.logq_backward(env, sp_b, wts)
        g1.record()
        torch.cuda.synchronize()
        bw_ms = g0.elapsed_time(g1)
        bw_flops = 3 * algorithmic_flops(inst) * B
        smmax_t = float(load_peaks()[0].get("sm_max_mhz", 2070.0))
        peak_t = 152 * 128 * 2 * smmax_t * 1e6 / 1e12
        del sp_b
        tuning = {"steps": args.tune_steps, "seconds": round(tune_s, 3),
                  "acceptance_first3": round(statistics.mean(h["acceptance"] for h in hist[:3]), 5),
                  "acceptance_last3": round(statistics.mean(h["acceptance"] for h in hist[-3:]), 5),
                  "kept_steps": sum(1 for h in hist if h["kept"]),
                  "backward_ms": round(bw_ms, 3),
                  "backward_roofline": {"bound": "alu", "unit": "TFLOP/s",
                                        "achieved": round(bw_flops / (bw_ms / 1e3) / 1e12, 3),
                                        "peak": round(peak_t, 3),
                                        "frac": round(bw_flops / (bw_ms / 1e3) / 1e12 / peak_t, 5),
                                        "flop_per_launch": bw_flops,
                                        "note": "3x the forward's algorithmic FLOPs (recompute + reverse sweeps)"}}

    spins = torch.empty((B, inst.Ly, inst.Lx), dtype=torch.int8, device=dev)
    logq = torch.empty(B, dtype=torch.float64, device=dev)
    energy = torch.empty(B, dtype=torch.float64, device=dev)
    flags = torch.empty(B, dtype=torch.int32, device=dev)
    acc = torch.empty(B, dtype=torch.uint8, device=dev)
    nacc = torch.zeros(1, dtype=torch.int64, device=dev)
    chain = Bd.init_chains(env, C, seed=args.seed + 7919 * rank, precision=prec)
    stream = torch.cuda.current_stream()
    l2_bytes = 126 * (1 << 20)
    out_bytes = spins.numel()
    flush = None if out_bytes > 2 * l2_bytes else torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_m = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]

    def step(i, timed):
        off = replicas.sample_offset(rank, world, i, B)
        if flush is not None:
            flush.fill_(i & 0xFF)
        if timed:
            ev_s[i].record(stream)
        Bd.sample(env, B, seed=args.seed, sample_offset=off, precision=prec,
                  out=(spins, logq, energy, flags), stream=stream)
        if timed:
            ev_m[i].record(stream)
        Bd.mh_step(env, C, T, (spins, logq, energy), chain, seed=args.seed + 1,
                   step_offset=replicas.mh_step_offset(rank, world, i, T), accepted=acc, n_accepted=nacc,
                   stream=stream)
        if timed:
            ev_e[i].record(stream)

    for i in range(args.warmup):
        step(i, False)
    torch.cuda.synchronize()
    nacc.zero_()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    wall0 = time.time()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(args.steps):
        step(i, True)
    t_end.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    wall = time.time() - wall0
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    sample_ms = [ev_s[i].elapsed_time(ev_m[i]) for i in range(args.steps)]
    n_accepted = int(nacc.item())
    total_ms, n_accepted = replicas.reduce_timing(total_ms, n_accepted, pg, dev)
    status = env.status()

    # end-to-end through the public API with host buffers: chain states live in pinned
    # host memory; every step uploads them, samples, runs MH, and reads back the chain
    # states and the accept flags.
    hs = torch.empty((C, inst.Ly, inst.Lx), dtype=torch.int8, pin_memory=True)
    hlq = torch.empty(C, dtype=torch.float64, pin_memory=True)
    hE = torch.empty(C, dtype=torch.float64, pin_memory=True)
    hacc = torch.empty(B, dtype=torch.uint8, pin_memory=True)
    hs.copy_(chain[0].cpu()); hlq.copy_(chain[1].cpu()); hE.copy_(chain[2].cpu())
    dchain = (torch.empty_like(chain[0]), torch.empty_like(chain[1]), torch.empty_like(chain[2]))
    nacc_e = torch.zeros(1, dtype=torch.int64, device=dev)
    step_ms_guess = total_ms / max(1, args.steps)
    e2e_steps = 1 if step_ms_guess > 5000 else max(1, min(args.steps, 3))
    h2d = hs.numel() + 16 * C
    d2h = hs.numel() + 16 * C + B
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(e2e_steps):
        off = replicas.sample_offset(rank, world, args.steps + i, B)
        dchain[0].copy_(hs, non_blocking=True); dchain[1].copy_(hlq, non_blocking=True); dchain[2].copy_(hE, non_blocking=True)
        Bd.sample(env, B, seed=args.seed, sample_offset=off, precision=prec, out=(spins, logq, energy, flags), stream=stream)
        Bd.mh_step(env, C, T, (spins, logq, energy), dchain, seed=args.seed + 1,
                   step_offset=replicas.mh_step_offset(rank, world, args.steps + i, T),
                   accepted=acc, n_accepted=nacc_e, stream=stream)
        hs.copy_(dchain[0], non_blocking=True); hlq.copy_(dchain[1], non_blocking=True); hE.copy_(dchain[2], non_blocking=True)
        hacc.copy_(acc, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    e2e_acc = int(nacc_e.item())

    plain = None
    if prec != "f64" and world == 1 and not args.no_plain:
        plain = plain_f64_form(Bd, env, inst, args, dev, stream)
    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    peaks, peak_src = load_peaks()
    flops = algorithmic_flops(inst, args.gauge)
    kern_s = statistics.mean(sample_ms) / 1e3
    achieved_tf = flops * B / kern_s / 1e12
    smmax = float(peaks.get("sm_max_mhz", 2070.0))
    out_bytes_per_sample = inst.Lx * inst.Ly + 8 + 8 + 4      # spins + log q + energy + flag
    achieved_gbs = out_bytes_per_sample * B / kern_s / 1e9
    if prec == "bf16":
        # the contraction is the bound; the int8 spins are ~0.1% of HBM time
        peak = float(peaks["bf16_tflops_sustained"])
        roof = {"bound": "tensor", "unit": "TFLOP/s", "achieved": round(achieved_tf, 2), "peak": peak,
                "frac": round(achieved_tf / peak, 5), "flop_per_sample": flops,
                "peak_source": peak_src + " bf16_tflops_sustained (kernel inside a long step)",
                "hbm": {"achieved_gbs": round(achieved_gbs, 2), "peak_gbs": float(peaks["hbm_gbs"]),
                        "bytes_per_sample": out_bytes_per_sample}}
    elif prec == "f32":
        peak = 152 * 128 * 2 * smmax * 1e6 / 1e12
        roof = {"bound": "alu", "unit": "TFLOP/s", "achieved": round(achieved_tf, 3), "peak": round(peak, 3),
                "frac": round(achieved_tf / peak, 5), "flop_per_sample": flops,
                "peak_source": "FP32 FFMA: 152 SM x 128 lanes x 2 x %.0f MHz" % smmax}
    else:
        peak = 1.25
        roof = {"bound": "alu", "unit": "TFLOP/s", "achieved": round(achieved_tf, 3), "peak": peak,
                "frac": round(achieved_tf / peak, 5), "flop_per_sample": flops,
                "peak_source": "FP64 nominal 1.25 TFLOP/s"}
    traffic = None
    if prec == "bf16":
        # DRAM bytes (read + write) per proposal and row of the tensor-core kernel, from ncu on
        # the 16x256 chi = 64 strip (69.91 + 68.46 GB for 65536 proposals x 16 rows); the
        # right stack dominates it and grows in proportion to proposals x rows
        traffic = round(131_960.0 * B * inst.Ly)
    roof.update({"traffic": traffic, "kernel": "sample_%s" % prec, "kernel_ms": round(kern_s * 1e3, 3)})
    step_ms = total_ms / args.steps
    props_s = B * world / (step_ms / 1e3)
    acc_rate = n_accepted / (B * world * args.steps)
    value = n_accepted / (total_ms / 1e3)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.config, prec, args.cpu_seconds)
        if cpu is not None and cpu.get("value") is not None:
            # accepted/s: the oracle's own acceptance where it was measured, else this run's
            a_cpu = cpu.get("measured_acceptance")
            cpu["acceptance_used"] = "oracle's own" if a_cpu is not None else "this run's (oracle's unmeasured)"
            cpu["value"] = cpu["value"] * (a_cpu if a_cpu is not None else acc_rate)
            cpu["unit"] = "accepted samples/s"
    line = {
        "metric": "accepted samples/s (TNMH proposals + MH, %s)" % desc,
        "value": round(value, 3), "unit": "accepted samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_ms, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"f64": "f64", "f32": "f32", "bf16": "bf16"}[prec],
        "data": "synthetic (seeded instance generator)",
        "config": {"workload": args.config, "description": desc, "Lx": inst.Lx, "Ly": inst.Ly, "chi": inst.chi,
                   "beta": inst.beta, "B": B, "chains": C, "proposals_per_chain": T, "precision": prec,
                   "gauge": args.gauge,
                   "parallelism": "replicas%d" % world,
                   "l2": "flushed (256 MiB write between steps)" if flush is not None else "outputs > L2"},
        "proposals_per_s": round(props_s, 3), "acceptance": round(acc_rate, 5),
        "env_build_s": round(env_build_s, 3), "logZ": info["logZ"], "device_status": status,
        "tuning": tuning,
        "roofline": roof, "cpu_baseline": cpu, "plain_f64": plain,
        "e2e": {"value": round(e2e_acc / (e2e_ms * e2e_steps / 1e3), 3) if e2e_ms > 0 else None,
                "unit": "accepted samples/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": round(e2e_ms, 3)},
        "gpu_launches": 3 * args.steps,
        "clocks": clk, "wall_s": round(wall, 3),
    }
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def run_batched_mixed(args):
    """Config 3 with the sampler chosen per chi class (batched.MixedRunner): chi < tc_chi on
    the persistent FP32 plan, chi >= tc_chi on the BF16 tensor-core sampler, one stream per
    instance, all concurrent.  Timed region: K steps, CUDA events on the current stream."""
    import torch
    from paper_2104_13264_gb300 import batched, instances

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    fac, Bdef, Cdef, pdef, desc = CONFIGS["c3"]
    insts = instances.config3()
    B = args.batch or Bdef
    C = args.chains or Cdef
    t0 = time.time()
    run = batched.MixedRunner(insts, B, C, tc_chi=args.tc_chi, seed=args.seed + 7919 * rank)
    build_s = time.time() - t0
    for _ in range(args.warmup):
        run.step()
    torch.cuda.synchronize()
    run.reset_counts()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        run.step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    sec = e0.elapsed_time(e1) / 1e3
    acc = run.n_accepted()
    props = B * len(insts) * args.steps
    flops = sum(algorithmic_flops(i) for i in insts) * B * args.steps
    ach = flops / sec / 1e12
    peaks, peak_src = load_peaks()
    peak = peaks["bf16_tflops_sustained"]
    if rank != 0:
        return
    line = {
        "metric": "accepted samples/s (TNMH proposals + MH, %s)" % desc, "value": round(acc / sec * world, 3),
        "unit": "accepted samples/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(sec / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (chi < %d) + bf16 (chi >= %d)" % (args.tc_chi, args.tc_chi),
        "data": "synthetic (seeded Gaussian couplings)",
        "config": {"workload": "c3", "description": desc, "instances": len(insts), "B": B, "chains": C,
                   "tc_chi": args.tc_chi, "tensor_core_instances": len(run.big_idx),
                   "fp32_instances": len(run.small_idx), "form": "per-chi-class samplers on concurrent streams"},
        "acceptance": round(acc / props, 5), "proposals_per_s": round(props / sec * world, 3),
        "flagged_fraction": run.flagged_fraction(), "env_build_s": round(build_s, 3),
        "roofline": {"bound": "tensor", "achieved": round(ach, 3), "peak": peak, "unit": "TFLOP/s",
                     "frac": round(ach / peak, 5), "traffic": None, "kernel": "whole step",
                     "peak_source": "bf16_tflops_sustained (%s)" % peak_src,
                     "note": "algorithmic FLOPs of every instance over the whole step time, against the sustained "
                             "BF16 peak (most of the work is on the tensor cores)"},
        "cpu_baseline": None, "e2e": None, "clocks": clk,
        "gpu_launches": (2 * len(run.big_idx) + 4) * args.steps,
    }
    print(json.dumps(line), flush=True)


def run_batched(args):
    """The batched persistent form: every instance's proposals in one persistent launch,
    the MH scan of every chain in one launch, both replayed from a captured CUDA graph;
    tiles and item order from the autotuner.  Timed region: K graph replays."""
    import torch
    from paper_2104_13264_gb300 import batched
    from paper_2104_13264_gb300 import binding as Bd
    from paper_2104_13264_gb300 import instances, replicas

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    fac, Bdef, Cdef, pdef, desc = CONFIGS["c3"]
    insts = instances.config3()
    B = args.batch or Bdef
    C = args.chains or Cdef
    prec = args.precision or pdef
    dev = torch.device("cuda", local)
    t0 = time.time()
    envs = Bd.build_envs_batched(insts, precisions=tuple(sorted({"f64", prec})))
    statuses = [e.status() for e in envs]
    env_build_s = time.time() - t0
    t0 = time.time()
    run = batched.BatchRunner(envs, B, chains=C, precision=prec, seed=args.seed + 7919 * rank)
    tune_s = time.time() - t0
    plan = run.plan
    binf = plan.info()
    stream = torch.cuda.current_stream()
    run.capture()
    for _ in range(args.warmup):
        run.step()
    torch.cuda.synchronize()
    run.n_accepted.zero_()
    # one timed kernel-only launch of the persistent sampler for the roofline
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(args.steps):
        run.step()
    t_end.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    n_accepted = int(run.n_accepted.sum().item())
    props = binf["proposal_rows"]
    # kernel time of the persistent sampler alone (same launch, eager, events on its stream)
    ks = []
    for i in range(max(1, args.steps)):
        k0.record(stream)
        plan.sample(run.prop, stream=stream)
        k1.record(stream)
        torch.cuda.synchronize()
        ks.append(k0.elapsed_time(k1))
    kern_s = statistics.mean(ks) / 1e3
    balance, makespan_ms = plan.balance()      # of the last of these launches
    total_ms, n_accepted = replicas.reduce_timing(total_ms, n_accepted, pg, dev)

    # end to end: chain states of every instance uploaded from pinned host memory before,
    # and read back with the accept flags after, each graph replay
    hs = torch.empty_like(run.chain[0], device="cpu").pin_memory()
    hlq = torch.empty_like(run.chain[1], device="cpu").pin_memory()
    hE = torch.empty_like(run.chain[2], device="cpu").pin_memory()
    hacc = torch.empty_like(run.accepted, device="cpu").pin_memory()
    hs.copy_(run.chain[0]); hlq.copy_(run.chain[1]); hE.copy_(run.chain[2])
    nacc0 = int(run.n_accepted.sum().item())
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(1, min(args.steps, 5))
    e0.record(stream)
    for i in range(e2e_steps):
        run.chain[0].copy_(hs, non_blocking=True); run.chain[1].copy_(hlq, non_blocking=True)
        run.chain[2].copy_(hE, non_blocking=True)
        run.step()
        hs.copy_(run.chain[0], non_blocking=True); hlq.copy_(run.chain[1], non_blocking=True)
        hE.copy_(run.chain[2], non_blocking=True); hacc.copy_(run.accepted, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    e2e_acc = int(run.n_accepted.sum().item()) - nacc0
    h2d = hs.numel() + 16 * binf["chain_rows"]
    d2h = h2d + props

    plain = None
    if world == 1 and not args.no_plain:
        plain = plain_batched_f64(Bd, envs, insts, B, C, args, stream)
    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    flops = sum(algorithmic_flops(inst) for inst in insts) * B
    peaks, peak_src = load_peaks()
    smmax = float(peaks.get("sm_max_mhz", 2070.0))
    achieved_tf = flops / kern_s / 1e12
    if prec == "f32":
        peak = 152 * 128 * 2 * smmax * 1e6 / 1e12
        psrc = "FP32 FFMA: 152 SM x 128 lanes x 2 x %.0f MHz" % smmax
    else:
        peak, psrc = 1.25, "FP64 nominal 1.25 TFLOP/s"
    roof = {"bound": "alu", "unit": "TFLOP/s", "achieved": round(achieved_tf, 3), "peak": round(peak, 3),
            "frac": round(achieved_tf / peak, 5), "traffic": None, "kernel": "sample_batched_kernel",
            "kernel_ms": round(kern_s * 1e3, 3), "flop_per_launch": flops, "peak_source": psrc}
    step_ms = total_ms / args.steps
    acc_rate = n_accepted / (props * world * args.steps)
    value = n_accepted / (total_ms / 1e3)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline("c3", prec, args.cpu_seconds)
        if cpu is not None and cpu.get("value") is not None:
            cpu["value"] = cpu["value"] * acc_rate       # the oracle runs random tensors here
            cpu["acceptance_used"] = "this run's (oracle's unmeasured)"
            cpu["unit"] = "accepted samples/s"
    line = {
        "metric": "accepted samples/s (TNMH proposals + MH, %s)" % desc,
        "value": round(value, 3), "unit": "accepted samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_ms, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic (seeded instance generator)",
        "config": {"workload": "c3", "description": desc, "instances": len(insts), "B_per_instance": B,
                   "chains_per_instance": C, "precision": prec, "tile": plan.tile, "order": plan.order,
                   "grid": binf["grid"], "parallelism": "replicas%d" % world,
                   "l2": "outputs %.0f MB per step (spins + log q + energy)" % ((binf["proposal_bytes"] + 20 * props) / 1e6)},
        "proposals_per_s": round(props * world / (step_ms / 1e3), 3), "acceptance": round(acc_rate, 5),
        "flagged_fraction": float((run.prop[3] != 0).double().mean().item()),
        "load_balance": {"efficiency": round(balance, 4), "makespan_ms": round(makespan_ms, 3),
                         "definition": "sum of the CTAs' busy time / (grid x makespan) of one persistent launch, "
                                       "from per-CTA global-timer stamps"},
        "env_build_s": round(env_build_s, 3), "autotune_s": round(tune_s, 3),
        "device_status_nonzero": sum(1 for s in statuses if s),
        "roofline": roof, "cpu_baseline": cpu, "plain_f64": plain,
        "e2e": {"value": round(e2e_acc / (e2e_ms * e2e_steps / 1e3), 3) if e2e_ms > 0 else None,
                "unit": "accepted samples/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": round(e2e_ms, 3)},
        "gpu_launches": 5 * args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def run_equilibration(args):
    """The paper's equilibration test (Sec. 3, Table hb) on the batched form: every
    iteration draws one proposal per chain (one persistent launch), runs the MH scan,
    one checkerboard Metropolis sweep of every chain and the forced log q of the new
    chain states, all replayed from one captured CUDA graph.  Reports iterations/s and
    the Delta diagnostic (eq. Delta) after each iteration of a fresh run."""
    import torch
    from paper_2104_13264_gb300 import batched
    from paper_2104_13264_gb300 import binding as Bd
    from paper_2104_13264_gb300 import instances

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    fac, Bdef, Cdef, pdef, desc = CONFIGS["c3d"]
    insts = instances.gaussian_ea_batch()
    C = args.chains or Cdef
    T = max(1, (args.batch or Bdef) // C)
    prec = args.precision or pdef
    stream = torch.cuda.current_stream()
    t0 = time.time()
    envs = Bd.build_envs_batched(insts, precisions=tuple(sorted({"f64", prec})))
    statuses = [e.status() for e in envs]
    env_build_s = time.time() - t0
    run = batched.BatchRunner(envs, C * T, chains=C, precision=prec, tile=64, order="cost", tune=False,
                              seed=args.seed + 7919 * rank, sweeps=1)
    run.capture()
    # Delta after each iteration of a fresh run (the first graph replay is iteration 1)
    deltas = [run.delta()[0]]
    for _ in range(args.iters):
        run.step()
        deltas.append(run.delta()[0])
    reached = {}
    for thr in TABLE_HB["thresholds"]:
        hit = next((k for k, d in enumerate(deltas) if abs(d) < thr), None)
        reached[str(thr)] = hit
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        run.step()
    torch.cuda.synchronize()
    run.n_accepted.zero_()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        run.step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = e0.elapsed_time(e1)
    props = len(insts) * C * T
    acc = int(run.n_accepted.sum().item()) / (props * args.steps)
    if rank != 0:
        return
    # algorithmic work per iteration: the proposals and the forced evaluation of the chains
    flops = sum(algorithmic_flops(i) for i in insts) * C * (T + 1)
    it_s = args.steps / (total_ms / 1e3)
    peaks, _ = load_peaks()
    smmax = float(peaks.get("sm_max_mhz", 2070.0))
    if prec == "f32":
        peak, psrc = 152 * 128 * 2 * smmax * 1e6 / 1e12, "FP32 FFMA nominal: 152 SM x 128 lanes x 2 x %.0f MHz" % smmax
    else:
        peak, psrc = 1.25, "FP64 nominal 1.25 TFLOP/s"
    achieved = flops * it_s / 1e12
    line = {
        "metric": "TNMH + Metropolis iterations/s (%s)" % desc, "value": round(it_s, 3), "unit": "iterations/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": prec, "data": "synthetic (seeded Gaussian couplings)",
        "config": {"workload": "c3d", "description": desc, "instances": len(insts), "L": 32, "T": 0.212, "chi": 16,
                   "chains_per_instance": C, "proposals_per_chain_per_iteration": T, "metropolis_sweeps": 1,
                   "precision": prec, "l2": "working set < L2 (graph replays back to back)"},
        "acceptance": round(acc, 5), "env_build_s": round(env_build_s, 3),
        "device_status_nonzero": sum(1 for s_ in statuses if s_),
        "delta_trajectory": [round(d, 5) for d in deltas],
        "iterations_to_delta": reached, "paper_table_hb": TABLE_HB,
        "roofline": {"bound": "alu", "unit": "TFLOP/s", "achieved": round(achieved, 4), "peak": peak,
                     "frac": round(achieved / peak, 5), "traffic": None, "kernel": "whole iteration",
                     "flop_per_iteration": flops, "peak_source": psrc},
        "cpu_baseline": None, "e2e": None, "gpu_launches": 6 * args.steps, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_frozen(args):
    """Closed lattices by frozen lines (App. B, Table hbpbc): every move freezes a random
    row and column of each torus, builds one environment per chain for the open lattice
    left (one batched builder launch), draws the proposals of the free spins (one
    persistent launch), evaluates the current free spins and runs the MH scan.  Reports
    moves/s (wall clock: the host assembles the open instances) and Delta per move."""
    import torch
    from paper_2104_13264_gb300 import frozen, instances

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    fac, Bdef, Cdef, pdef, desc = CONFIGS["c3p"]
    Jh, Jv, h, beta = instances.gaussian_ea_torus_batch()
    C = args.chains or Cdef
    prec = args.precision or pdef
    D, L = Jh.shape[0], Jh.shape[1]
    start = np.random.default_rng([args.seed, 19]).choice([-1, 1], size=(D, C, L, L)).astype(np.int8)
    ch = frozen.FrozenLineChains(Jh, Jv, h, beta, 16, start, precision=prec, proposals=1, seed=args.seed + 7919 * rank)
    deltas = [ch.delta()[0]]
    acc, walls = [], []
    for _ in range(args.iters):
        torch.cuda.synchronize()
        t0 = time.time()
        a = ch.step()
        torch.cuda.synchronize()
        walls.append(time.time() - t0)
        acc.append(a.float().mean().item())
        deltas.append(ch.delta()[0])
    if rank != 0:
        return
    reached = {str(t): next((k for k, d in enumerate(deltas) if abs(d) < t), None) for t in TABLE_HBPBC["thresholds"]}
    timed = walls[args.warmup:] or walls
    per = statistics.mean(timed)
    line = {
        "metric": "frozen-line TNMH moves/s (%s)" % desc, "value": round(1.0 / per, 4), "unit": "moves/s",
        "n_gpus": world, "steps": len(timed), "warmup": min(args.warmup, len(walls)),
        "ms_per_step": round(per * 1e3, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": prec, "data": "synthetic (seeded Gaussian couplings)",
        "config": {"workload": "c3p", "description": desc, "disorders": D, "L": L, "T": 0.212, "chi": 16,
                   "chains_per_disorder": C, "proposals_per_chain_per_move": 1, "cuts": "random row and column",
                   "environments_per_move": D * C, "timing": "wall clock per move (host cut + GPU work)"},
        "acceptance": round(float(np.mean(acc)), 5), "delta_trajectory": [round(d, 5) for d in deltas],
        "iterations_to_delta": reached, "paper_table_hbpbc": TABLE_HBPBC,
        "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None,
    }
    print(json.dumps(line), flush=True)


def _compress_dims_flops(dl, pp, dr, kmax):
    """Bond dims after the successive SVD of an MPS (QR sweep: min(dl p, dr); SVD sweep:
    min(kmax, dl, p dr)) and the FLOPs of its projections and absorptions (the Jacobi
    sweeps of the factorisations are not counted)."""
    dl, dr = list(dl), list(dr)
    n = len(dl)
    fl = 0
    for i in range(n - 1):
        length, b = dl[i] * pp[i], dr[i]
        k = min(length, b)
        fl += 2 * k * b * length + 2 * k * b * pp[i + 1] * dr[i + 1]
        dr[i], dl[i + 1] = k, k
    for i in range(n - 1, 0, -1):
        a, length = dl[i], pp[i] * dr[i]
        k = min(kmax, a, length)
        fl += 2 * a * k * length + 2 * dl[i - 1] * pp[i - 1] * a * k
        dl[i], dr[i - 1] = k, k
    return dl, dr, fl


def cube_contraction_flops(dims, chi):
    """FLOPs per 3D proposal of the sampler's contractions (bottom and top boundary
    products, the sandwich vectors R and Lambda, the site weights) and of the QR/SVD
    projections of its boundary compressions, from the layer PEPS dims [Lz, Ly, Lx, 4].
    The iterative Jacobi sweeps are left out, so this is a lower bound of the work."""
    Lz, Ly, Lx, _ = dims.shape
    fl = 0
    for z in range(Lz):
        d = dims[z]
        bot = [None] * Ly
        bot[Ly - 1] = [1] * (Lx + 1)
        for y in range(Ly - 2, -1, -1):
            dl, pp, dr = [], [], []
            for x in range(Lx):
                du, dlx, dd, drx = (int(v) for v in d[y + 1, x])
                bl, br = bot[y + 1][x], bot[y + 1][x + 1]
                fl += 3 * du * dlx * dd * drx + 2 * (dlx * bl) * du * (drx * br) * dd
                dl.append(dlx * bl)
                pp.append(du)
                dr.append(drx * br)
            dl2, _, f = _compress_dims_flops(dl, pp, dr, chi)
            fl += f
            bot[y] = dl2 + [1]
        tb = [1] * (Lx + 1)
        for y in range(Ly):
            for x in range(Lx):
                du, dlx, dd, drx = (int(v) for v in d[y, x])
                ta, tc, pb, qb = tb[x], tb[x + 1], bot[y][x], bot[y][x + 1]
                if x > 0:
                    fl += 2 * ta * du * drx * qb * tc + 2 * ta * dlx * dd * qb * du * drx + 2 * ta * dlx * pb * dd * qb
                fl += (2 * dlx * pb * du * tc * ta + 2 * dlx * du * tc * dd * qb * pb + 2 * dlx * du * dd * drx * tc * qb
                       + 4 * du * dlx * dd * drx + 2 * tc * drx * qb * dlx * du * dd)
            if y + 1 < Ly:
                dl, pp, dr = [], [], []
                for x in range(Lx):
                    du, dlx, dd, drx = (int(v) for v in d[y, x])
                    fl += 2 * (tb[x] * dlx) * dd * (tb[x + 1] * drx) * du
                    dl.append(tb[x] * dlx)
                    pp.append(dd)
                    dr.append(tb[x + 1] * drx)
                dl2, _, f = _compress_dims_flops(dl, pp, dr, chi)
                fl += f
                tb = dl2 + [1]
    return fl


def run_cube(args):
    """Three-dimensional TNMH (Sec. 3D): the 16^3 ferromagnet with layer PEPS of bond D and
    boundary MPS of bond chi; a step is B proposals (one thread each) and the MH scan of C
    chains over them."""
    import torch
    from paper_2104_13264_gb300 import binding as Bd
    from paper_2104_13264_gb300 import instances

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fac, Bdef, Cdef, pdef, desc = CONFIGS["c6"]
    if args.cube_model == "afm":
        inst = instances.cubic_antiferromagnet(L=args.cube_L, T=args.cube_T, D=args.cube_D, chi=args.cube_chi)
        desc = desc.replace("ferromagnet", "antiferromagnet in a field h=3")
    else:
        inst = instances.cubic_ferromagnet(L=args.cube_L, T=args.cube_T, D=args.cube_D, chi=args.cube_chi)
    desc = desc.replace("T=4.5", "T=%g" % args.cube_T).replace("D=2, chi=2", "D=%d, chi=%d" % (inst.D, inst.chi))
    B = args.batch or Bdef
    C = args.chains or Cdef
    T = B // C
    B = C * T
    prec = args.precision or pdef
    stream = torch.cuda.current_stream()
    t0 = time.time()
    env = Bd.Env3D.from_instance(inst, gauge=args.gauge)
    build_s = time.time() - t0
    assert env.status() == 0, "3D build reported a numerical problem"
    chain = Bd.init_chains3d(env, C, seed=args.seed + 1, precision=prec)
    nacc = torch.zeros(1, dtype=torch.int64, device=dev)
    acc_hist = []

    def step(k):
        sp, lq, E, fl = Bd.sample3d(env, B, seed=args.seed, sample_offset=(rank << 40) + k * B, precision=prec)
        a = Bd.mh_step3d(env, C, T, (sp, lq, E), chain, seed=args.seed + 2, step_offset=(rank << 40) + k * T,
                         n_accepted=nacc)
        return a

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    nacc.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(args.steps):
        acc_hist.append(step(args.warmup + k))
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    sec = e0.elapsed_time(e1) / 1e3
    acc = int(nacc.item())
    acceptance = acc / (B * args.steps)
    # end to end: the same steps with the accepted count read back every step
    t1 = time.time()
    for k in range(args.steps):
        step(args.warmup + args.steps + k)
        _ = int(nacc.item())
    e2e_s = time.time() - t1
    # the plain FP64 form on a bounded subset
    plain = None
    if not args.no_plain:
        nb = min(B, 2048)
        Bd.sample3d(env, 128, seed=args.seed, precision="f64")
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        Bd.sample3d(env, nb, seed=args.seed, sample_offset=1 << 41, precision="f64")
        p1.record(stream)
        torch.cuda.synchronize()
        ps = p0.elapsed_time(p1) / 1e3
        plain = {"proposals": nb, "proposals_per_s": round(nb / ps, 3), "precision": "f64"}
    dims = env.export()["dims"]
    flops = cube_contraction_flops(dims, inst.chi)
    ach = flops * B * args.steps / sec / 1e12
    peak = 152 * 128 * 2 * 2070e6 / 1e12 if prec == "f32" else 1.25
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import peps3d
        build = peps3d.build_env3d_bond if args.gauge == "bond" else peps3d.build_env3d
        oenv = build(inst.Jx, inst.Jy, inst.Jz, inst.h, inst.beta, inst.D, inst.chi)
        nb = 32
        c0 = time.time()
        peps3d.sample3d(oenv, nb, seed=args.seed)
        cs = time.time() - c0
        cpu = {"value": round(nb * acceptance / cs, 4), "unit": "accepted samples/s", "cores": 1, "kind": "oracle",
               "sample": "%d proposals of the same 16^3 workload drawn by the numpy oracle (vectorised over samples, "
                         "one process), times the GPU chains' acceptance" % nb,
               "proposals_per_s": round(nb / cs, 4)}
    if rank != 0:
        return
    value = acc / sec * world
    line = {
        "metric": "accepted samples/s (3D TNMH proposals + MH, %s)" % desc, "value": round(value, 3),
        "unit": "accepted samples/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(sec / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": prec, "data": "synthetic (uniform couplings)",
        "config": {"workload": "c6", "description": desc, "model": inst.name, "L": args.cube_L, "T": args.cube_T,
                   "gauge": args.gauge, "D": inst.D,
                   "chi": inst.chi, "B": B, "chains": C, "proposals_per_chain": T,
                   "multi_gpu": "replicas only: each rank runs its own chains"},
        "acceptance": round(acceptance, 5), "env_build_s": round(build_s, 3),
        "roofline": {"bound": "alu", "achieved": round(ach, 4), "peak": round(peak, 3), "unit": "TFLOP/s",
                     "frac": round(ach / peak, 5), "traffic": None, "kernel": "sample3d_kernel<%s>" % prec,
                     "flop_per_sample": flops,
                     "peak_source": "FP32 FFMA nominal: 152 SM x 128 lanes x 2 x 2070 MHz" if prec == "f32"
                     else "FP64 nominal 1.25 TFLOP/s",
                     "flop_note": "contractions and QR/SVD projections counted from the layer dims; the iterative "
                                  "Jacobi sweeps are not counted (lower bound)"},
        "cpu_baseline": cpu, "plain_f64": plain, "clocks": clk,
        "e2e": {"value": round(acc / e2e_s * world, 3), "unit": "accepted samples/s",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 8},
        "gpu_launches": (2 + 2) * args.steps,
    }
    print(json.dumps(line), flush=True)


def plain_batched_f64(Bd, envs, insts, B, C, args, stream):
    """The plain FP64 form of the batched workload: one tnmc_sample + tnmc_mh_step per
    instance, FP64, no graph, default tiles."""
    import torch
    dev = torch.device("cuda")
    T = B // C
    outs = (torch.empty(B * max(e.Lx * e.Ly for e in envs), dtype=torch.int8, device=dev),
            torch.empty(B, dtype=torch.float64, device=dev), torch.empty(B, dtype=torch.float64, device=dev),
            torch.empty(B, dtype=torch.int32, device=dev))
    chains = [Bd.init_chains(e, C, seed=args.seed + 3, precision="f64") for e in envs]
    nacc = torch.zeros(1, dtype=torch.int64, device=dev)

    def one_pass(k):
        for i, e in enumerate(envs):
            sp = outs[0][:B * e.Lx * e.Ly].view(B, e.Ly, e.Lx)
            Bd.sample(e, B, seed=args.seed, sample_offset=(i << 40) + k * B, precision="f64",
                      out=(sp, outs[1], outs[2], outs[3]), stream=stream)
            Bd.mh_step(e, C, T, (sp, outs[1], outs[2]), chains[i], seed=args.seed + 5, step_offset=(i << 40) + k * T,
                       n_accepted=nacc, stream=stream)

    one_pass(0)
    torch.cuda.synchronize()
    nacc.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    one_pass(1)
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    acc = int(nacc.item())
    n = B * len(envs)
    return {"proposals": n, "chains": C * len(envs), "proposals_per_s": round(n / sec, 3),
            "accepted_per_s": round(acc / sec, 3), "acceptance": round(acc / n, 5), "seconds": round(sec, 3)}


def plain_f64_form(Bd, env, inst, args, dev, stream):
    """The plain FP64 SIMT form on a bounded subset of the same workload: proposals/s,
    and accepted samples/s with its own MH scan (chains of the same length T)."""
    import torch
    n = max(256, int(args.plain_batch))
    T = min(n, max(1, (args.batch or CONFIGS[args.config][1]) // (args.chains or CONFIGS[args.config][2])))
    C = max(1, n // T)
    n = C * T
    out = (torch.empty((n, inst.Ly, inst.Lx), dtype=torch.int8, device=dev),
           torch.empty(n, dtype=torch.float64, device=dev), torch.empty(n, dtype=torch.float64, device=dev),
           torch.empty(n, dtype=torch.int32, device=dev))
    Bd.sample(env, 128, seed=args.seed, precision="f64", out=tuple(x[:128] for x in out), stream=stream)
    chain = Bd.init_chains(env, C, seed=args.seed + 3, precision="f64")
    nacc = torch.zeros(1, dtype=torch.int64, device=dev)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    Bd.sample(env, n, seed=args.seed, sample_offset=1 << 40, precision="f64", out=out, stream=stream)
    Bd.mh_step(env, C, T, out[:3], chain, seed=args.seed + 5, n_accepted=nacc, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    acc = int(nacc.item())
    return {"proposals": n, "chains": C, "proposals_per_s": round(n / sec, 3),
            "accepted_per_s": round(acc / sec, 3), "acceptance": round(acc / n, 5), "seconds": round(sec, 3)}


def _oracle_workload(config, n_rows_cap):
    """Oracle environment for timing: the real one when cheap, else random tensors with
    the configuration's bond dimensions for the first rows (the oracle's cost does not
    depend on the tensor values)."""
    import numpy as np

    from oracle import tnmc
    from paper_2104_13264_gb300 import instances
    fac = CONFIGS[config][0]
    inst = getattr(instances, fac)()
    if config in ("c3", "c3d"):
        # a cost-weighted sample: one of the largest instances (L = 64, chi = 32) stands for
        # the mean by the ratio of algorithmic work, applied by the caller
        insts = inst
        big = max(insts, key=lambda i: algorithmic_flops(i))
        rows = min(big.Ly, n_rows_cap)
        rng = np.random.default_rng(0)
        env = tnmc.Env(big.Lx, rows, big.beta, big.chi, big.Jh[:rows], big.Jv[:rows - 1], big.h[:rows])
        for r in range(rows):
            env.M[r] = [rng.standard_normal((tnmc.bond_dim(big.chi, big.Lx, big.Ly, r, c), 2,
                                             tnmc.bond_dim(big.chi, big.Lx, big.Ly, r, c + 1))) ** 2
                        for c in range(big.Lx)]
        mean_flops = sum(algorithmic_flops(i) for i in insts) / len(insts)
        scale = algorithmic_flops(big) / mean_flops
        return env, big, rows, ("random positive tensors with the bond dimensions of the first %d rows of a "
                                "%dx%d chi=%d instance, rate scaled by %.3f to the batch's mean work per proposal"
                                % (rows, big.Ly, big.Lx, big.chi, scale)), scale
    if inst.Lx * inst.Ly <= 4096:
        env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi)
        return env, inst, inst.Ly, "oracle-built environment", 1.0
    rows = min(inst.Ly, n_rows_cap)
    rng = np.random.default_rng(0)
    env = tnmc.Env(inst.Lx, rows, inst.beta, inst.chi, inst.Jh[:rows], inst.Jv[:rows - 1], inst.h[:rows])
    for r in range(rows):
        env.M[r] = [rng.standard_normal((tnmc.bond_dim(inst.chi, inst.Lx, inst.Ly, r, c), 2,
                                         tnmc.bond_dim(inst.chi, inst.Lx, inst.Ly, r, c + 1))) ** 2
                    for c in range(inst.Lx)]
    return env, inst, rows, "random positive tensors with the bond dimensions of the first %d rows" % rows, 1.0


def host_cores():
    """Cores this process may run on (the affinity mask; the machine may have more)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


_W_ENV = None


def _oracle_init(env):
    global _W_ENV
    _W_ENV = env


def _oracle_job(job):
    """One oracle worker's share: C chains of T proposals drawn with the oracle sampler
    (sample indices from `offset`), then, when `mh`, each chain's random start and its MH
    scan.  Returns (proposals, accepted or None, seconds)."""
    from oracle import tnmc
    C, T, seed, offset, mh, beta = job
    t0 = time.time()
    sp, lq, E, _ = tnmc.sample(_W_ENV, C * T, seed=seed, sample_offset=offset)
    acc = None
    if mh:
        cs, clq, cE = tnmc.init_chains(_W_ENV, C, seed + 1)
        a, _, _, _ = tnmc.mh_scan(beta, C, T, sp, lq, E, cs, clq, cE, seed=seed + 2, step_offset=offset)
        acc = int(a.sum())
    return C * T, acc, time.time() - t0


class OraclePool:
    """The FP64 oracle on `workers` host processes (spawn start method, one numpy thread
    each), every worker holding the same environment; a round gives each worker whole
    chains, so the union of the rounds is the oracle's own chain over more proposals."""

    def __init__(self, env, beta, workers, mh):
        import multiprocessing as mp
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        self.workers, self.beta, self.mh = workers, beta, mh
        self.pool = mp.get_context("spawn").Pool(workers, initializer=_oracle_init, initargs=(env,))
        self.offset = 0

    def round(self, per_worker, seed=0):
        C = max(1, per_worker // 16)
        T = max(1, per_worker // C)
        jobs = []
        for _ in range(self.workers):
            jobs.append((C, T, seed, self.offset, self.mh, self.beta))
            self.offset += C * T
        t0 = time.time()
        res = self.pool.map(_oracle_job, jobs)
        wall = time.time() - t0
        props = sum(r[0] for r in res)
        acc = sum(r[1] for r in res) if self.mh else None
        return props, acc, wall

    def calibrate(self, seconds):
        """Proposals per worker for a round of about `seconds`."""
        n = 1
        while True:
            _, _, wall = self.round(n)
            if wall > seconds / 4 or n >= (1 << 16):
                break
            n *= 4
        return max(1, min(1 << 16, int(n * seconds / max(wall, 1e-3))))

    def close(self):
        self.pool.terminate()
        self.pool.join()


def cpu_baseline(config, prec, seconds):
    """The oracle on the host cores, in a child process without the GPU: all-core and
    single-core rates on a bounded sample (see _cpu_rate)."""
    code = ("import sys, json; sys.path.insert(0, %r); import bench; print(json.dumps(bench._cpu_rate(%r, %r)))"
            % (ROOT, config, float(seconds)))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    try:
        p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
        return json.loads(p.stdout.strip().splitlines()[-1])
    except Exception as e:  # noqa: BLE001
        return {"value": None, "error": str(e)[-200:]}


def _cpu_rate(config, seconds):
    """Oracle proposals/s (and accepted/s where its own environment is affordable) on all
    usable host cores, and on one core, each timed for about seconds / 2."""
    env, inst, rows, how, wscale = _oracle_workload(config, 4)
    real = rows == inst.Ly and how.startswith("oracle")
    scale = inst.Ly / rows / wscale
    out = {"kind": "oracle", "unit": "proposals/s"}
    for label, workers in (("single_core", 1), ("all_cores", host_cores())):
        pool = OraclePool(env, inst.beta, workers, real)
        try:
            per = pool.calibrate(seconds / 2)
            props, acc, wall = pool.round(per)
        finally:
            pool.close()
        out[label] = {"cores": workers, "proposals": props, "seconds": round(wall, 3),
                      "proposals_per_s": props / (wall * scale),
                      "acceptance": (acc / props) if real else None}
    a = out["all_cores"]
    out.update({"value": a["proposals_per_s"], "cores": a["cores"],
                "measured_acceptance": a["acceptance"],
                "sample": "%d proposals of %s over %d of %d rows (%s)%s; numpy, one thread per process, "
                          "%d processes" % (a["proposals"], config, rows, inst.Ly, how,
                                            ", rate scaled to the full lattice" if scale != 1 else "",
                                            a["cores"])})
    return out


def run_reference(args):
    """The FP64 oracle timed on the host cores as the reference arm (rank 0 only).

    Each step is one round of the oracle on every usable host core (spawned processes,
    one numpy thread each, whole chains per process): draw a bounded batch of proposals
    and, where the oracle's own environment is affordable (n <= 4096 sites), run the MH
    scan of each process's chains, so accepted samples/s is measured.  On the 256 x 256
    lattice the oracle cannot build the environment in minutes; it is then timed on
    random tensors with the bond dimensions of the first rows, its acceptance is not
    known, and its proposals/s (an upper bound of accepted samples/s) is reported with
    the per-row extrapolation stated in its own field.  `ms_per_step` is the wall time of
    the work each step actually ran.
    """
    world, rank, local = dist_setup(args)
    if rank != 0:
        return
    env, inst, rows, how, wscale = _oracle_workload(args.config, 4)
    fac, Bdef, Cdef, pdef, desc = CONFIGS[args.config]
    real = rows == inst.Ly and how.startswith("oracle")
    workers = host_cores()
    pool = OraclePool(env, inst.beta, workers, real)
    try:
        per = args.cpu_batch if args.cpu_batch > 0 else pool.calibrate(4.0)
        for _ in range(args.warmup):
            pool.round(per)
        props, acc, walls = 0, 0, []
        for _ in range(args.steps):
            p_, a_, w_ = pool.round(per)
            props += p_
            acc += a_ or 0
            walls.append(w_)
    finally:
        pool.close()
    total = sum(walls)
    scale = inst.Ly / rows / wscale
    unit = "accepted samples/s"
    if real:
        value, note = acc / (total * scale), None
    else:
        value = props / (total * scale)
        note = "oracle proposals/s on random tensors of the right shapes: an upper bound of accepted samples/s"
    cpu = {"value": round(value, 6), "unit": unit, "cores": workers, "kind": "oracle",
           "sample": "%d proposals per step over %d of %d rows (%s), %d processes"
                     % (props // max(1, args.steps), rows, inst.Ly, how, workers),
           "acceptance": (acc / props) if real else None}
    if note:
        cpu["note"] = note
    line = {"impl": "reference", "metric": "accepted samples/s (TNMH proposals + MH, %s)" % desc,
            "value": round(value, 6), "unit": unit, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total / max(1, args.steps) * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded instance generator)",
            "config": {"workload": args.config, "description": desc,
                       "proposals_per_step": props // max(1, args.steps)},
            "extrapolation": None if scale == 1 else {
                "rows_run": rows, "rows_total": inst.Ly, "work_scale": round(wscale, 6),
                "rate_divided_by": round(scale, 6),
                "note": "each step samples the first rows only; the oracle's cost per row does not depend on "
                        "the tensor values, so the rate is divided by this factor"},
            "cpu_baseline": cpu,
            "e2e": {"value": round(value, 6), "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tnmc", choices=["tnmc", "reference"])
    ap.add_argument("--config", default=os.environ.get("TNMC_BENCH_CONFIG", "c5"), choices=sorted(CONFIGS))
    ap.add_argument("--precision", default=None, choices=["f64", "f32", "bf16"])
    ap.add_argument("--batch", type=int, default=None)
    ap.add_argument("--chains", type=int, default=None)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--cpu-batch", type=int, default=0)
    ap.add_argument("--plain-batch", type=int, default=2 * 152 * 64)   # one full wave of the FP64 kernel
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--iters", type=int, default=30, help="iterations of the Delta trajectory (c3d)")
    ap.add_argument("--gauge", default=None, choices=["spin", "bond"],
                    help="environment gauge: spin basis, or the bond basis of App. A (2D: chi <= 32; 3D: 2 D chi <= 64)")
    ap.add_argument("--tc-chi", type=int, default=0,
                    help="config 3: instances with chi >= this use the BF16 tensor-core sampler (0: all FP32 batched)")
    ap.add_argument("--cube-L", type=int, default=16, help="3D lattice side (c6)")
    ap.add_argument("--cube-T", type=float, default=4.5, help="3D temperature (c6)")
    ap.add_argument("--cube-D", type=int, default=2, help="3D layer PEPS bond (c6)")
    ap.add_argument("--cube-chi", type=int, default=2, help="3D boundary MPS bond (c6)")
    ap.add_argument("--cube-model", default="ferro", choices=["ferro", "afm"],
                    help="3D model: ferromagnet, or antiferromagnet in a field h = 3 (c6)")
    ap.add_argument("--tune-steps", type=int, default=0,
                    help="tuning steps of the FP32 tensors before the timed sampling (the 64x64 Villain case uses 50)")
    args = ap.parse_args()
    if args.gauge is None:
        # the 3D line runs the bond basis (the form that reaches the paper's 3D acceptance)
        args.gauge = "bond" if args.config == "c6" else "spin"
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "c3" and args.tc_chi:
        run_batched_mixed(args)
    elif args.config == "c3":
        run_batched(args)
    elif args.config == "c3d":
        run_equilibration(args)
    elif args.config == "c3p":
        run_frozen(args)
    elif args.config == "c6":
        run_cube(args)
    else:
        run_tnmc(args)


if __name__ == "__main__":
    main()
