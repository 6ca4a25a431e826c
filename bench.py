"""Benchmark of the batched rigid-body step on GB300.

Workload (one bench step): one persistent forward rollout of the 9-body
quadruped, 65,536 environments x 1,000 steps (10 substeps each), synthetic
seeded inputs resident in HBM; when the adjoint is available, the same
rollout's reverse pass follows and is timed as the fwd+bwd figure.

Prints one JSON line (rank 0).  `value` = forward env-steps/s over all ranks.
The roofline is FP32-ALU bound: achieved = algorithmic flops per launch (the
oracle's flop count per env-step, stored in paper_2106_13281_gb300/data) /
the kernel's CUDA-event duration; peak = 152 SMs x 128 FP32 lanes x 2 flops
x 2.07 GHz.

`--impl reference` times the FP64 oracle (the reference arm of this method:
a plain CPU program) on a bounded sample of the same workload on the host
cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "env-steps/s fwd and fwd+bwd, 9-body quadruped @64k envs; % roofline; err vs FP64"
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12  # 80.54


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--envs", type=int, default=65536)
    p.add_argument("--horizon", type=int, default=1000, help="steps per rollout")
    p.add_argument("--checkpoint-every", type=int, default=0,
                   help="K of the fwd+bwd figure (0: picked by the autotuner)")
    p.add_argument("--no-autotune", action="store_true", help="keep the default launch configuration")
    p.add_argument("--bwd-variant", type=int, default=-1,
                   help="reverse-kernel launch-bounds variant 0..3 (default: the autotuner's or the smallest that fits)")
    p.add_argument("--e2e-first-steps", type=int, default=16,
                   help="first chunk of the streamed (e2e) rollout; later chunks double up to 250 steps")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-secondary", action="store_true",
                   help="skip the other configurations (biped, adjoint, heterogeneous batch) in the headline run")
    p.add_argument("--workload", default="quadruped", choices=["quadruped", "biped", "adjoint", "hetero"],
                   help="quadruped: the headline line; the others time the remaining configurations "
                        "(biped forward 16384 x 1000; quadruped adjoint 4096 x 100 and x 1000; heterogeneous "
                        "batch fwd+bwd 65536 x 200) and print one informational line each")
    return p.parse_args()


def headline_config(N, T, substeps, dt, A, world):
    """The workload both arms report (the reference arm times a bounded sample
    of it, described in its cpu_baseline.sample)."""
    return {"workload": f"quadruped-9body forward rollout, {N} envs x {T} steps x {substeps} substeps",
            "envs": N, "steps_per_rollout": T, "substeps": substeps, "dt": dt,
            "l2": "inputs larger than L2 (actions %.2f GB per rollout)" % (N * T * A * 4 / 1e9),
            "parallelism": f"env shards x{world}"}


# The translation unit of the forward kernels (the dominant kernel of the
# headline): its .cu file and the headers of csrc/ it includes.
FORWARD_TU = ("brax_device.cuh", "brax_forward.cu", "brax_kernels.h", "brax_pair.cuh", "brax_params.h",
              "brax_physics.cuh")


def kernel_sources_digest():
    """sha256 over the forward kernels' sources (FORWARD_TU, in that order):
    a change there invalidates a recorded DRAM-traffic capture, a change of
    the host code around them does not."""
    import hashlib
    d = os.path.join(ROOT, "paper_2106_13281_gb300", "csrc")
    h = hashlib.sha256()
    for n in FORWARD_TU:
        h.update(n.encode())
        with open(os.path.join(d, n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic(key, path=None):
    """The small-case ncu capture of the dominant kernel recorded in
    data/traffic.json under `key`, or None when the kernel sources changed
    since (the counters then describe another kernel)."""
    p = path or os.path.join(ROOT, "paper_2106_13281_gb300", "data", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f).get(key)
    if not rec or rec.get("sources_sha256") != kernel_sources_digest():
        return None
    return rec


def scaled_traffic(rec, T, n_chunks, state_bytes):
    """DRAM bytes of one full launch of T steps, scaled from a small capture
    of the same kernel (rec: its steps, DRAM reads and the state bytes of its
    environments).  The capture's reads beyond the initial state are the
    per-step stream (the actions), which grows with the steps; the state is
    read once and written once per chunk of the chunked schedule (a later
    chunk's state was evicted from L2 by the actions streamed in between), so
    reads = T x per-step + state x chunks and writes = state x chunks."""
    per_step = (rec["dram_read_bytes"] - rec["state_bytes"]) / rec["steps"]
    chunks = max(1, int(n_chunks))
    return int(round(T * per_step + 2 * state_bytes * chunks))


def alg_flops(scene="quadruped"):
    with open(os.path.join(ROOT, "paper_2106_13281_gb300", "data", "alg_flops.json")) as f:
        return json.load(f)[scene]


class Clocks:
    """Sample SM clocks and throttle reasons with nvidia-smi during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world, local


def barrier_max(x, world):
    """Maximum of a per-rank time over all ranks (timing only; no data-path collective)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_seed(rank):
    """Each rank simulates its own shard of environments (weak scaling)."""
    return 1 + 1000 * rank


def aggregate_rate(world, envs_per_rank, steps_per_rollout, rollouts, max_ms):
    """Whole-job env-steps/s: every rank's env-steps over the slowest rank's time."""
    return world * envs_per_rank * steps_per_rollout * rollouts / (max_ms / 1e3)


def run_ours(args):
    import numpy as np
    import torch

    from paper_2106_13281_gb300 import scenes as S
    from paper_2106_13281_gb300.system import BraxSystem

    rank, world, local = dist_setup(args.gpus)
    N, T = args.envs, args.horizon
    d = S.quadruped()
    sysm = BraxSystem(d)
    seed = shard_seed(rank)
    rp, rr, ang = S.initial_conditions(d, N, seed, height_jitter=0.05)
    f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    state0 = sysm.default_qp(N, f32(rp), f32(rr), f32(ang))
    actions = f32(S.actions(d, N, T, seed))
    state_T = torch.empty_like(state0)
    stream = torch.cuda.current_stream()
    # launch configuration and checkpoint interval: picked by timing the
    # workload itself (brax_autotune), before any timed region
    tuning = {"autotuned": not args.no_autotune}
    if args.bwd_variant >= 0:  # a fixed reverse-kernel launch (profiling runs without the autotuner)
        from paper_2106_13281_gb300.binding import check as check_rc
        check_rc(sysm._L.brax_system_set_backward_launch(sysm.handle, args.bwd_variant))
        tuning["bwd_variant"] = args.bwd_variant
    K = args.checkpoint_every if args.checkpoint_every > 0 else 10
    if not args.no_autotune:
        r = sysm.autotune(state0, actions)
        tuning.update(fwd_kernel="two_envs_per_thread" if r["fwd_kernel"] else "one_env_per_thread",
                      fwd_groups=r["fwd_groups"], fwd_variant=r["fwd_variant"], fwd_candidates=r["n_candidates"])
        if args.checkpoint_every <= 0:
            # (the reverse candidates are timed on the first 16384 environments)
            rr_ = sysm.autotune(state0, actions, reverse=True, forward=False)
            K = rr_["K"]
            tuning.update(K=K, bwd_variant=rr_["bwd_variant"], reverse_sample_envs=min(N, 16384))

    def step():
        sysm.rollout(state0, actions, state_T=state_T)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sysm.sync_status()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        start.record(stream)
        for e0, e1 in ev:
            e0.record(stream)
            step()
            e1.record(stream)
        end.record(stream)
        torch.cuda.synchronize()
    sysm.sync_status()
    launch = sysm.last_rollout()
    total_ms = barrier_max(start.elapsed_time(end), world)
    kern_ms = statistics.mean(e0.elapsed_time(e1) for e0, e1 in ev)
    envsteps = N * T
    value = aggregate_rate(world, N, T, args.steps, total_ms)

    # end to end through the public API: pinned host inputs in, state back out, every step
    h_state0 = state0.cpu().pin_memory()
    h_actions = actions.cpu().pin_memory()
    h_out = torch.empty_like(h_state0).pin_memory()

    # the actions stream in on a copy stream in chunks (16 steps, doubling up
    # to 250) while the previous chunk runs (brax_rollout_streamed)
    e2e_bufs = {}
    e2e_chunk, e2e_first = 250, args.e2e_first_steps

    def e2e_step():
        return sysm.rollout_streamed(h_state0, h_actions, h_out, chunk_steps=e2e_chunk, bufs=e2e_bufs,
                                     first_steps=e2e_first)

    e2e_launches = e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = barrier_max(e0.elapsed_time(e1), world)
    e2e_value = aggregate_rate(world, N, T, args.steps, e2e_ms)
    h2d = h_state0.numel() * 4 + h_actions.numel() * 4
    d2h = h_out.numel() * 4

    # forward + reverse pass of the same workload (checkpoints every K steps)
    gT = torch.zeros_like(state0)
    gT[:, 0, 0] = -1.0  # d/dstate_T of -(torso x displacement)
    ckpt = torch.empty((math.ceil(T / K), N, sysm.B, 13), device="cuda", dtype=torch.float32)
    ws = torch.empty((sysm.workspace_size(N, T, K),), device="cuda", dtype=torch.uint8)
    g_actions = torch.empty_like(actions)
    g_state0 = torch.empty_like(state0)
    L = sysm._L
    from paper_2106_13281_gb300.binding import _ptr, check

    def fwd_bwd():
        check(L.brax_rollout(sysm.handle, N, T, K, _ptr(state0), _ptr(actions), _ptr(state_T), _ptr(ckpt), None, None,
                             stream.cuda_stream))
        check(L.brax_rollout_backward(sysm.handle, N, T, K, _ptr(state0), _ptr(actions), _ptr(ckpt), _ptr(gT), None,
                                      _ptr(g_actions), _ptr(g_state0), _ptr(ws), ws.numel(), stream.cuda_stream))

    fb_steps = max(1, min(args.steps, 3))
    for _ in range(max(1, min(args.warmup, 2))):
        fwd_bwd()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(fb_steps):
        fwd_bwd()
    f1.record(stream)
    torch.cuda.synchronize()
    sysm.sync_status()
    fb_ms = barrier_max(f0.elapsed_time(f1), world)
    fwd_bwd_value = aggregate_rate(world, N, T, fb_steps, fb_ms)
    del ws, ckpt

    # state read and written once, actions read once (the per-launch algorithmic bytes)
    algorithmic_bytes = 2 * state0.numel() * 4 + actions.numel() * 4
    # DRAM traffic of the timed launch, scaled from the small-case capture of the same kernel
    rec = measured_traffic(f"quadruped_pair_{N}") if world == 1 else None
    traffic, traffic_note = None, "no capture of the current kernel sources"
    if rec is not None and tuning.get("fwd_kernel", "two_envs_per_thread") == "two_envs_per_thread":
        traffic = scaled_traffic(rec, T, launch["n_chunks"], state0.numel() * 4)
        traffic_note = (f"scaled from one ncu capture of {rec['kernel']} at {N} envs x {rec['steps']} steps "
                        f"(dram read {rec['dram_read_bytes']} B, write {rec['dram_write_bytes']} B) to "
                        f"{T} steps in {max(1, launch['n_chunks'])} chunk(s)")
    fl = alg_flops("quadruped")
    flops_per_envstep = fl["flops_per_env_step"]
    achieved_tflops = flops_per_envstep * envsteps / (kern_ms / 1e3) / 1e12
    # forward + reverse: the forward, one forward recompute and the tape's reverse-op count
    fb_flops = 2 * flops_per_envstep + fl["reverse_flops_per_env_step"]
    fb_tflops = fb_flops * envsteps / (fb_ms / fb_steps / 1e3) / 1e12
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "env-steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded PCG64 actions uniform[-1,1], initial joint angles N(0,0.1^2), heights 0.75+U(0,0.05))",
        "config": headline_config(N, T, int(d["substeps"]), float(d["dt"]), d["gear"].shape[0], world),
        "e2e": {"value": e2e_value, "unit": "env-steps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "api": "brax_rollout_streamed (C ABI; pinned host state and actions in, state out; chunks of %d "
                       "steps doubling to %d on the system's copy stream, overlapped with compute)"
                       % (min(e2e_first, e2e_chunk), e2e_chunk),
                "gpu_launches_per_step": e2e_launches},
        "gpu_launches": args.steps,
        "fwd_bwd": {"value": fwd_bwd_value, "unit": "env-steps/s", "steps": fb_steps, "checkpoint_every": K,
                    "ms_per_step": fb_ms / fb_steps, "gpu_launches": 2 * fb_steps,
                    "roofline": {"bound": "alu", "achieved": fb_tflops, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                                 "frac": fb_tflops / FP32_PEAK_TFLOPS, "flops_per_env_step": fb_flops,
                                 "note": "forward + one forward recompute + the oracle tape's reverse-op count"},
                    "loss": "-(torso x displacement); gradients w.r.t. the action sequence and the initial state"},
        "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved_tflops / FP32_PEAK_TFLOPS,
                     "traffic": traffic, "traffic_note": traffic_note,
                     "algorithmic_bytes": algorithmic_bytes,
                     "peak_note": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz",
                     "flops_per_env_step": flops_per_envstep, "kernel_ms": kern_ms},
        "clocks": clk.summary(),
        "tuning": dict(tuning, launch=launch),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(d, sysm, seed)
    if rank == 0 and world == 1 and not args.no_secondary:
        # the other configurations of the method, timed in the same run
        with Clocks(local) as clk2:
            other = {w: workload_lines(args, w) for w in ("biped", "adjoint", "hetero")}
        line["configs_other"] = dict(other, clocks=clk2.summary())
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def cpu_baseline(d, sysm, seed, n_envs=2048, T=200):
    """The FP64 oracle on a bounded sample of the same workload (host cores),
    plus the GPU's one-step position error against it on that sample."""
    import numpy as np
    import torch

    from oracle import oracle as orc
    from paper_2106_13281_gb300 import scenes as S
    rp, rr, ang = S.initial_conditions(d, n_envs, seed, height_jitter=0.05)
    st = orc.default_qp(d, n_envs, rp, rr, ang).astype(np.float32).astype(np.float64)
    a = S.actions(d, n_envs, T, seed).astype(np.float64)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    ref = orc.rollout(d, st, a, n_threads=cores)
    dt = time.perf_counter() - t0
    one = orc.rollout(d, st, a[:1], n_threads=cores)
    f32 = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    got = sysm.rollout(f32(st), f32(a[:1]))["state_T"].cpu().numpy()
    err = float(np.abs(got[..., :3] - one[..., :3]).max())
    return {"value": n_envs * T / dt, "unit": "env-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_envs} envs x {T} steps of the same quadruped workload (seed {seed}), FP64, "
                      f"{cores} threads", "err_vs_fp64_1step_max_m": err}


def run_reference(args):
    """The FP64 oracle as the reference arm: each step is a bounded sample
    (1024 envs x 100 steps) of the quadruped workload on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np

    from oracle import oracle as orc
    from paper_2106_13281_gb300 import scenes as S
    d = S.quadruped()
    n_envs, T = 1024, 100
    rp, rr, ang = S.initial_conditions(d, n_envs, 1, height_jitter=0.05)
    st = orc.default_qp(d, n_envs, rp, rr, ang)
    a = S.actions(d, n_envs, T, 1).astype(np.float64)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        orc.rollout(d, st, a, n_threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orc.rollout(d, st, a, n_threads=cores)
    dt = time.perf_counter() - t0
    value = n_envs * T * args.steps / dt
    sample = f"{n_envs} envs x {T} steps of the quadruped workload per step, FP64 oracle, {cores} threads"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": headline_config(args.envs, args.horizon, int(d["substeps"]), float(d["dt"]), d["gear"].shape[0],
                                  args.gpus),
        "cpu_baseline": {"value": value, "unit": "env-steps/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "env-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def _timed(fn, warmup, steps):
    """Mean ms of fn over `steps` runs after `warmup` runs (CUDA events on the
    current stream, synchronised on both sides)."""
    import torch
    for _ in range(max(3, warmup)):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_workload(args):
    """One other configuration of the method (--workload), one JSON line per
    figure (not the headline)."""
    for ln in workload_lines(args, args.workload):
        print(json.dumps(ln), flush=True)


def workload_lines(args, workload):
    """The other configurations of the method: biped forward, quadruped
    adjoint (100 and 1,000 steps), heterogeneous batch fwd+bwd; a list of
    result dicts."""
    import numpy as np
    import torch

    from paper_2106_13281_gb300 import scenes as S
    from paper_2106_13281_gb300.system import BraxBatch, BraxSystem
    f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    steps = max(1, min(args.steps, 3))

    def setup(name, N, T, seed, drop=0.0):
        d = S.SCENES[name]()
        sysm = BraxSystem(d)
        rp, rr, ang = S.initial_conditions(d, N, seed, height_jitter=0.05)
        rp[:, 2] -= drop
        return d, sysm, sysm.default_qp(N, f32(rp), f32(rr), f32(ang)), f32(S.actions(d, N, T, seed))

    def roof(flops_per_envstep, envsteps, ms):
        t = flops_per_envstep * envsteps / (ms / 1e3) / 1e12
        return {"bound": "alu", "achieved": t, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": t / FP32_PEAK_TFLOPS, "flops_per_env_step": flops_per_envstep}

    lines = []
    if workload == "biped":
        N, T = 16384, 1000
        d, sysm, st, a = setup("biped", N, T, 2)
        r = sysm.autotune(st, a)
        out = torch.empty_like(st)
        ms = _timed(lambda: sysm.rollout(st, a, state_T=out), args.warmup, steps)
        sysm.sync_status()
        lines.append({"metric": "env-steps/s fwd, 17-body biped (self-collision) @16k envs", "value": N * T / ms * 1e3,
                      "unit": "env-steps/s", "ms_per_step": ms, "steps": steps,
                      "config": {"workload": "biped-17body forward rollout, 16384 envs x 1000 steps x 10 substeps"},
                      "roofline": roof(alg_flops("biped")["flops_per_env_step"], N * T, ms),
                      "tuning": {k: r[k] for k in ("fwd_kernel", "fwd_groups", "fwd_variant")}})
    elif workload == "adjoint":
        for T in (100, 1000):
            N = 4096
            d, sysm, st, a = setup("quadruped", N, T, 3, drop=0.0)
            r = sysm.autotune(st, a, reverse=True)
            K = r["K"]
            gT = torch.zeros_like(st)
            gT[:, 0, 0] = -1.0
            ws = torch.empty((sysm.workspace_size(N, T, K),), device="cuda", dtype=torch.uint8)
            out = torch.empty_like(st)

            def fb2():
                o = sysm.rollout(st, a, K=K, checkpoints=True, state_T=out)
                sysm.rollout_backward(st, a, o["checkpoints"], gT, None, K=K, workspace=ws)

            ms = _timed(fb2, args.warmup, steps)
            sysm.sync_status()
            fq = alg_flops("quadruped")
            lines.append({"metric": "env-steps/s fwd+bwd, 9-body quadruped adjoint @4096 envs",
                          "value": N * T / ms * 1e3, "unit": "env-steps/s", "ms_per_step": ms, "steps": steps,
                          "roofline": roof(2 * fq["flops_per_env_step"] + fq["reverse_flops_per_env_step"], N * T, ms),
                          "config": {"workload": f"quadruped adjoint, 4096 envs x {T} steps, loss -torso x "
                                                 "displacement (+ action penalty, differentiated by torch)",
                                     "checkpoint_every": K},
                          "tuning": {k: r[k] for k in ("K", "bwd_variant", "fwd_bwd_ms_per_step")}})
            del ws
    else:  # heterogeneous batch, forward + reverse in one launch each
        names, ns, T = ["pendulum", "quadruped", "biped", "arm_box"], [32768, 16384, 8192, 8192], 200
        descs = [S.SCENES[n]() for n in names]
        systems = [BraxSystem(dd) for dd in descs]
        sts, acs, gts = [], [], []
        for i, (dd, sy, n) in enumerate(zip(descs, systems, ns)):
            rp, rr, ang = S.initial_conditions(dd, n, 4 + i, height_jitter=0.05)
            st = sy.default_qp(n, f32(rp), f32(rr), f32(ang))
            sts.append(st.reshape(-1))
            acs.append(f32(S.actions(dd, n, T, 4 + i)).reshape(-1))
            g = torch.zeros_like(st)
            g[:, -1 if names[i] == "arm_box" else (len(dd["parent"]) if names[i] == "pendulum" else 0), 0] = -1.0
            gts.append(g.reshape(-1))
        batch = BraxBatch(systems, ns)
        st, a, gT = torch.cat(sts), torch.cat(acs), torch.cat(gts)
        K = 10
        warps, _ = batch.autotune(st, a, T, K=K, reverse=True)
        ws = torch.empty((batch.workspace_size(T, K),), device="cuda", dtype=torch.uint8)

        def fwd():
            return batch.rollout(st, a, T, K=K, checkpoints=True)

        def fb():
            o = fwd()
            batch.rollout_backward(st, a, o["checkpoints"], gT, T, K=K, workspace=ws)

        ms_f = _timed(fwd, args.warmup, steps)
        # forward + reverse captured in one CUDA graph (two kernel nodes), replayed
        for _ in range(2):
            fb()
        torch.cuda.synchronize()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            with torch.cuda.graph(graph, stream=side):
                fb()
        torch.cuda.current_stream().wait_stream(side)
        ms = _timed(graph.replay, args.warmup, steps)
        fl = sum(alg_flops(n)["flops_per_env_step"] * k for n, k in zip(names, ns)) / sum(ns)
        lines.append({"metric": "env-steps/s fwd+bwd, heterogeneous batch (one launch each way)",
                      "value": sum(ns) * T / ms * 1e3, "unit": "env-steps/s", "ms_per_step": ms, "steps": steps,
                      "fwd_only": {"value": sum(ns) * T / ms_f * 1e3, "ms_per_step": ms_f,
                                   "roofline": roof(fl, sum(ns) * T, ms_f)},
                      "config": {"workload": "32768 pendulum + 16384 quadruped + 8192 biped + 8192 arm+box, "
                                             "200 steps, checkpoints every 10", "checkpoint_every": K},
                      "tuning": {"warps_per_block": warps}, "cuda_graph": True})
    for ln in lines:
        ln.update({"n_gpus": 1, "warmup": args.warmup, "dtype": "f32", "data": "synthetic", "higher_is_better": True})
    return lines


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "quadruped":
        run_workload(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
