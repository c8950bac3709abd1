"""Benchmark of the in-hand tracking hot path on one GB300 (or N replicas).

A step is one tracking window of Algorithm 1 over N environments: T = 10
frames, each a batched simulation step (kinematic hand, narrowphase, Jacobi
contact solve, integration, sensor pads) followed by the FP64 cost and the
argmin estimate, then one optimizer update (elite-weighted resample and
perturbation). The default workload is the N = 1024 tracking loop (cylinder
of 64 spheres, 4 fingers x 4 capsule links + palm, 8 pads, 20 Jacobi
iterations, 2 substeps at 30 Hz). Inputs are seeded and synthetic.

Output: one JSON line (metric env-steps/s: environment-frames advanced per
second including cost, argmin and the amortised optimizer update).
  --impl ours        the CUDA path through libinhand.so (default)
  --impl reference   the FP64 CPU oracle on the same workload (bounded sample,
                     one thread per host core)
Besides the main line (with the step kernel's FP32 roofline against the
measured FMA throughput of the GPU, and the end-to-end rate through the C ABI
from pinned host buffers), a single-GPU run also measures the uneven batch
(N = 8192, shapes of 16-256 spheres, 10/20/40 iterations), the mug sweep
(N = 1024 ... 32768, forward and forward + adjoint) with a bounded search for
the largest N that holds 30 tracking frames/s, the forward + adjoint of a
30-frame horizon (N = 1024), the PD-driven hand's window, and the oracle on
the host cores. The paper's studies (optimizer comparison, cost-term
ablation, warm start, refined vs plain tracking) run with --part.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic FP32 operations of the step, counted from the kernel's source
# (an FMA counts as 2; an add, multiply, compare, min/max, select, sqrt,
# rsqrt, division, sin or cos as 1), attached to the work counters the step
# kernel reports (pairs tested after culling, contacts, contact-iterations,
# env-substeps, env-iterations with contacts, (link, cluster) tests):
#   env-substep   gravity 3, rotation matrix 39, world inverse inertia 81,
#                 integration with the rotation exponential 61; link cull 25
#                 per link, cluster centre to world 15 per cluster, sphere
#                 centre to world 15 per sphere
#   pair tested   sphere to link frame, closest point, gap and normal 34,
#                 lever arm 6, contact test 1
#   cluster test  offset 3, reach of the link's bounding capsule 25
#   contact       r x n 9, k_n 21, tr K 29, inverses 3, bias 4, target
#                 velocity 6, lever arm and pad membership 10, pad sum 9
#                 (a finger contact's link point velocity, 108 more, is not
#                 counted: the counters do not tell palm and finger apart)
#   contact-iter  relative velocity 15, normal and tangential components and
#                 steps 31, disk clamp 13, relaxation 15 (update_contact, 74);
#                 its moment 9 and the impulse and moment sums 6
#   env-iter      body velocity from the summed impulses and moments 24
FLOP_PER_ENV_SUBSTEP = 184     # + 25 per link + 15 per cluster (flops_of)
FLOP_PER_LINK = 25
FLOP_PER_CLUSTER = 15
FLOP_PER_SPHERE = 15
FLOP_PER_PAIR = 41
FLOP_PER_CLUSTER_TEST = 28
FLOP_PER_CONTACT = 91
FLOP_PER_CONTACT_ITER = 89
FLOP_PER_ENV_ITER = 24
# DRAM traffic of one step_kernel launch (dram__bytes_read.sum +
# dram__bytes_write.sum) from the ncu capture summarised in
# profiles/step_kernel_tracking_cyl64.md, valid for the step kernel's own
# sources (step.cu, step_kernel.cuh, contact.cuh) whose hash is recorded with it; reported as
# null once they change.
STEP_TRAFFIC = {"bytes_per_launch": 200192, "sources_sha256": "91521be734c85a5a59a84b2be37a4cf619b2a3268b2665d3306d11e1368d318d"}
STEP_SOURCES = ["paper_2002_12160_gb300/csrc/step.cu", "paper_2002_12160_gb300/csrc/step_kernel.cuh",
                "paper_2002_12160_gb300/csrc/contact.cuh"]


def step_sources_sha():
    import hashlib
    h = hashlib.sha256()
    for f in STEP_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def step_traffic():
    if STEP_TRAFFIC["bytes_per_launch"] is None or STEP_TRAFFIC["sources_sha256"] != step_sources_sha():
        return None
    return STEP_TRAFFIC["bytes_per_launch"]


# bytes of HBM traffic per env-frame the step must move: state in/out
# (pose, vel 64 B each way), params (8 B), shape/iters/status (12 B), forces
STATE_BYTES_PER_ENV = 64 + 64 + 8 + 12 + 4


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="tracking_cyl64")
    p.add_argument("--n-envs", type=int, default=None)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--main-only", action="store_true",
                   help="only the main line (no uneven batch, mug sweep, largest-N search, adjoint, PD hand)")
    p.add_argument("--part", choices=["all", "adjoint", "optimizers", "warm", "pd", "pd_speed", "refine"],
                   default="all",
                   help="the paper's studies, outside the default line: adjoint throughput, optimizer "
                        "comparison, warm start, PD hand (with the cost-term ablation; pd_speed: throughput "
                        "only), refined vs plain update at equal wall time")
    p.add_argument("--shape", default=None, help="force the step kernel shape, e.g. 64x2 (default: autotune)")
    p.add_argument("--sweep", default=None,
                   help="comma-separated N values: also time the workload at each N (tracking frames/s)")
    return p.parse_args()


def hbm_peak():
    """HBM copy bandwidth measured on the GB300s (MEASURED_PEAKS.json),
    else the pool's earlier single measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured (MEASURED_PEAKS.json hbm_gbs: STREAM-style copy)"
    except (OSError, KeyError, ValueError, TypeError):
        return 6800.0, "fallback (an earlier copy measurement on a GB300)"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"inhand_clocks_gpu{gpu_index}_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- distributed
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """The largest of every rank's x (the slowest rank sets the job's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- reference arm
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_tracking_rate(workload, threads, budget_s, n_per_thread=16, n_frames=300, T=10, max_windows=None):
    """The FP64 oracle as it stands, tracking on the host: each of `threads`
    threads runs its own `n_per_thread` environments of the workload (its first
    `n_frames` frames replayed from fresh initial samples) through whole windows
    -- every frame the ground-truth environment's step (the observation), the
    samples' step and cost, then the optimizer -- until the time budget (or
    `max_windows` windows per thread) is spent. The oracle is C called through
    ctypes, which releases the interpreter lock, so the threads run on separate
    cores. Returns (env-steps/s of the samples, windows timed, frames per thread)."""
    import threading
    import oracle as O
    from paper_2002_12160_gb300 import workloads as W
    wl = W.make_workload(workload, n_envs=n_per_thread, frames=n_frames)
    osc = O.OracleScene(wl.scene)
    done = [0] * threads
    wins = [0] * threads
    deadline = [None]
    start = threading.Barrier(threads + 1)

    def worker(t):
        gt0 = wl.gt_pose if wl.gt_pose is not None else wl.nominal_pose
        upd = 0
        start.wait()
        while time.perf_counter() < deadline[0] and (max_windows is None or wins[t] < max_windows):
            pose, theta = O.sample_initial(n_per_thread, O.pose8_to7(wl.nominal_pose), wl.init,
                                           wl.seed + 1000 * t + upd)
            st = O.State(pose, np.zeros((n_per_thread, 6)), theta, wl.shape_id, wl.iters)
            gt = O.State(O.pose8_to7(gt0)[None], np.zeros((1, 6)), np.array([wl.theta_gt]))
            f = 0
            while f + T <= n_frames and time.perf_counter() < deadline[0] and \
                    (max_windows is None or wins[t] < max_windows):
                c_sum = np.zeros(n_per_thread)
                for k in range(T):
                    obs, _ = O.step(osc, wl.sim, gt, wl.q_traj, f, 1)
                    forces, _ = O.step(osc, wl.sim, st, wl.q_traj, f, 1)
                    _, c_mean, _ = O.cost(wl.sim, forces, obs[0], st.status, c_sum, k + 1)
                    f += 1
                    done[t] += 1
                O.optimizer(wl.opt, st, c_mean, wl.seed + t, upd)
                upd += 1
                wins[t] += 1

    th = [threading.Thread(target=worker, args=(t,), daemon=True) for t in range(threads)]
    for x in th:
        x.start()
    deadline[0] = time.perf_counter() + budget_s
    t0 = time.perf_counter()
    start.wait()
    for x in th:
        x.join()
    el = time.perf_counter() - t0
    return n_per_thread * sum(done) / el, sum(wins), done, el


def run_reference(args, rank, world):
    """The FP64 oracle as it stands on the host cores, on the workload our arm
    runs: whole tracking windows on a bounded sample of its environments (16
    per host core). Rank 0 alone runs it."""
    if rank != 0:
        return
    from paper_2002_12160_gb300 import workloads as W
    T = 10
    cores = host_cores()
    n_per = 16
    wl_full = W.make_workload(args.workload, n_envs=args.n_envs)
    # each timed step: one window per core; warm-up steps first
    _ = oracle_tracking_rate(args.workload, cores, 1e9, n_per_thread=n_per, max_windows=args.warmup)
    value, wins, done, el = oracle_tracking_rate(args.workload, cores, 1e9, n_per_thread=n_per,
                                                 max_windows=args.steps)
    ms = 1e3 * el / max(1, args.steps)
    sample = (f"{n_per} envs x {cores} threads (one per host core) of {args.workload}, whole {T}-frame windows "
              f"incl. each thread's ground-truth env and the optimizer; {args.steps} windows per thread timed "
              f"after {args.warmup} warm-up windows")
    line = {"impl": "reference", "metric": "env-steps/s", "value": value, "unit": "env-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "n_envs": wl_full.n_envs, "window_frames": T,
                       "links": wl_full.scene.n_links, "pads": wl_full.scene.n_pads,
                       "substeps": wl_full.sim.substeps, "parallelism": f"replicas{args.gpus}"},
            "cpu_baseline": {"value": value, "unit": "env-steps/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "env-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(workload, budget_s=8.0):
    """The oracle's tracking throughput on the host (env-steps/s), all host
    cores (one thread each) and one thread, each leg on a bounded sample."""
    cores = host_cores()
    multi, _, done_m, el_m = oracle_tracking_rate(workload, cores, budget_s)
    single, _, done_s, el_s = oracle_tracking_rate(workload, 1, budget_s)
    return {"value": multi, "unit": "env-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"16 envs per thread x {cores} threads of {workload}, {sum(done_m)} thread-frames in "
                      f"{el_m:.1f} s (first 300 frames replayed from fresh samples; windows of 10 incl. the "
                      f"ground-truth env's step, cost, optimizer)",
            "single_thread": {"value": single, "cores": 1,
                              "sample": f"16 envs, {done_s[0]} frames in {el_s:.1f} s"}}


# ----------------------------------------------------------------------------- our arm
def measure(workload, n_envs, steps, warmup, shape, rank, world, local, n_timing=3, n_e2e=0, tune_frames=4,
            adjoint_h=0):
    """Time `steps` tracking windows (graph replays) of a workload on this rank's
    GPU; then `n_timing` windows launched kernel by kernel (the step kernel's own
    time and work), `n_e2e` windows end to end from pinned host buffers, and
    (adjoint_h > 0) the forward + adjoint of an adjoint_h-frame horizon cost of
    every environment from the state reached (checkpoints every 10 frames)."""
    import torch
    from paper_2002_12160_gb300 import tracking, workloads as W
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    T = 10
    n_windows = warmup + steps + n_timing + n_e2e + (adjoint_h + T - 1) // T
    wl = W.make_workload(workload, n_envs=n_envs, frames=n_windows * T)
    seed = wl.seed + 7919 * rank   # independent replicas per rank
    tr = tracking.Tracker(wl, seed=seed)
    tr.prepare()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for w in range(warmup):
        tr.window(w)
    torch.cuda.synchronize()
    if shape:
        a, b = shape if isinstance(shape, tuple) else (int(v) for v in shape.lower().split("x"))
        tr.sim.sim_set_variant(a, b)
        chosen, tune_ms = (a, b), {}
    else:
        # pick the step kernel's shape on the frames after the warm-up windows, where
        # the contacts have settled (the autotuner restores the state after each trial)
        chosen, tune_ms = tr.sim.sim_autotune(warmup * T, tune_frames)
    torch.cuda.synchronize()
    tr.sim.sim_work_counters(reset=True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for s in range(steps):
            flush.zero_()
            ev[s][0].record(stream)
            tr.window(warmup + s)       # one captured graph: T fused steps + optimizer
            ev[s][1].record(stream)
        torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    ms = sum(ev[s][0].elapsed_time(ev[s][1]) for s in range(steps)) / steps
    work = tr.sim.sim_work_counters(reset=True)
    ms = max_over_ranks(ms, world)
    out = {"wl": wl, "n": tr.n, "T": T, "ms": ms, "work": work, "clocks": clk.summary(),
           "chosen": chosen, "tune_ms": tune_ms}
    w0 = warmup + steps
    if n_timing:
        # the dominant kernel alone: the same windows launched one kernel at a time,
        # every (fused) step bracketed by events on its stream, L2 flushed per window
        step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(n_timing)]
        tr.sim.sim_work_counters(reset=True)
        for s in range(n_timing):
            flush.zero_()
            tr.window_unfused(w0 + s, step_events=step_ev[s])
        torch.cuda.synchronize()
        out["work_t"] = tr.sim.sim_work_counters(reset=True)
        lst = [a.elapsed_time(b) for (a, b) in step_ev]
        out["step_ms"] = sum(lst) / len(lst)
        out["step_launches"] = n_timing
    if n_e2e:
        out["e2e"] = tr.e2e_windows(w0 + n_timing, n_e2e)
    if adjoint_h:
        f0 = (w0 + n_timing + n_e2e) * T
        obs = tr.obs[f0:f0 + adjoint_h].contiguous()
        tr.sim.sim_adjoint(f0, obs, checkpoint_every=min(10, adjoint_h))   # warm-up (sizes the scratch)
        torch.cuda.synchronize()
        lst = []
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            e0.record(stream)
            cost, grad, _ = tr.sim.sim_adjoint(f0, obs, checkpoint_every=min(10, adjoint_h))
            e1.record(stream)
            torch.cuda.synchronize()
            lst.append(e0.elapsed_time(e1))
        t = min(lst)
        out["adjoint"] = {"horizon": adjoint_h, "checkpoint_every": min(10, adjoint_h), "ms_per_call": t,
                          "env_steps_per_s": tr.n * adjoint_h / (t / 1e3),
                          "finite_envs": int(torch.isfinite(cost).sum().item())}
        del cost, grad
    out["add_mm"] = tr.add_mm()
    tr.close()
    del flush
    torch.cuda.empty_cache()
    return out


def measure_adjoint(local, n_envs=1024, horizon=30, checkpoint_every=10, reps=3, windows=4):
    """Forward + adjoint of the horizon cost (sim_adjoint) for every environment
    of the differentiable-tracking workload (box / cylinder, H = 30 frames,
    checkpoints every 10): CUDA-event time per call after one warm-up call.
    Then the refinement: `windows` tracking windows each followed by 3
    gradient steps on its elites, against as many plain windows (CUDA-event
    time per window, after one refined and one plain warm-up window)."""
    import torch
    from paper_2002_12160_gb300 import tracking, workloads as W
    torch.cuda.set_device(local)
    out = {}
    for name in ["tracking_cyl64", "tracking_box27"]:
        wl = W.make_workload(name, n_envs=n_envs, frames=20 + horizon + 2)
        tr = tracking.Tracker(wl, n_envs=n_envs)
        tr.prepare()
        for w in range(2):
            tr.window(w)          # contacts established, the population converging
        f0 = 20
        obs = tr.obs[f0:f0 + horizon].contiguous()
        tr.sim.sim_adjoint(f0, obs, checkpoint_every=checkpoint_every)   # warm-up (scratch)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = []
        for _ in range(reps):
            e0.record()
            cost, grad, _ = tr.sim.sim_adjoint(f0, obs, checkpoint_every=checkpoint_every)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        t = statistics.median(ms)
        fin = torch.isfinite(cost)
        out[name] = {"n_envs": n_envs, "horizon": horizon, "checkpoint_every": checkpoint_every,
                     "ms_per_call": t, "env_steps_per_s": n_envs * horizon / (t / 1e3),
                     "finite_envs": int(fin.sum().item()),
                     "mean_grad_norm": float(grad[fin].norm(dim=1).mean().item()) if fin.any() else None}
        tr.close()
        wl = W.make_workload(name, n_envs=n_envs, frames=10 * (2 * windows + 2))
        tr = tracking.Tracker(wl, n_envs=n_envs)
        tr.prepare()
        assert tr.T == 10
        tr.window_refined(0)
        tr.window(1)
        e2 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for w in range(2, 2 + windows):
            tr.window_refined(w)
        e1.record()
        for w in range(2 + windows, 2 + 2 * windows):
            tr.window(w)
        e2.record()
        torch.cuda.synchronize()
        ref_ms, plain_ms = e0.elapsed_time(e1) / windows, e1.elapsed_time(e2) / windows
        out[name]["refined_window"] = {"steps": 3, "elites": int(wl.opt.elite_frac * n_envs), "ms": ref_ms,
                                       "plain_window_ms": plain_ms, "ratio": ref_ms / plain_ms}
        tr.close()
    torch.cuda.empty_cache()
    return out


def refine_study(local, seeds=tuple(range(11, 35)), frames=300, n_refined=1024, steps=3):
    """Tracking error (ADD of the argmin estimate, mm, over `frames` frames) of
    the plain update against the update preceded by 3 gradient-refinement steps
    of the elites, at equal wall time: the refined run has N = n_refined; the
    plain run gets the N whose window takes as long (measured), and is also
    shown at N = n_refined. Median and mean over seeded trajectories."""
    import torch
    from paper_2002_12160_gb300 import tracking, workloads as W
    torch.cuda.set_device(local)

    def run(name, n, seed, refined, n_frames):
        wl = W.make_workload(name, n_envs=n, frames=n_frames, seed=seed)
        tr = tracking.Tracker(wl, n_envs=n)
        tr.prepare()
        nw = n_frames // tr.T
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for w in range(nw):
            if refined:
                tr.window_refined(w, steps=steps)
            else:
                tr.window(w)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / nw
        add = tr.add_mm(nw * tr.T)
        tr.close()
        return ms, add

    out = {}
    for name in ["tracking_cyl64", "tracking_box27"]:
        run(name, n_refined, seeds[0], True, 40)    # warm-up: scratch allocation, first captures
        ms_r = statistics.median(run(name, n_refined, seeds[0], True, 60)[0] for _ in range(2))
        # the plain window's time as a function of N; the equal-time N by interpolation
        grid = [1024, 2048, 4096, 8192, 16384, 32768]
        t_plain = [run(name, n, seeds[0], False, 60)[0] for n in grid]
        n_eq = grid[0]
        for a, b, ta, tb in zip(grid, grid[1:], t_plain, t_plain[1:]):
            if ta <= ms_r:
                n_eq = a if tb <= ta else int(a + (b - a) * min(1.0, (ms_r - ta) / (tb - ta)))
        n_eq = max(grid[0], min(grid[-1], 256 * (n_eq // 256)))
        res = {"refined": [], "plain_same_n": [], "plain_equal_time": []}
        times = {"refined": [], "plain_equal_time": []}
        for seed in seeds:
            ms, add = run(name, n_refined, seed, True, frames)
            res["refined"].append(add); times["refined"].append(ms)
            res["plain_same_n"].append(run(name, n_refined, seed, False, frames)[1])
            ms, add = run(name, n_eq, seed, False, frames)
            res["plain_equal_time"].append(add); times["plain_equal_time"].append(ms)
        out[name] = {
            "n_refined": n_refined, "n_plain_equal_time": n_eq, "refine_steps": steps, "frames": frames,
            "seeds": list(seeds),
            "ms_per_window": {k: statistics.median(v) for k, v in times.items()},
            "plain_ms_per_window_by_n": {str(n): t for n, t in zip(grid, t_plain)},
            "add_mm_median": {k: statistics.median(v) for k, v in res.items()},
            "add_mm_mean": {k: float(np.mean(v)) for k, v in res.items()},
            "add_mm": res,
            "refined_le_plain_equal_time": statistics.median(res["refined"]) <= statistics.median(res["plain_equal_time"])}
    torch.cuda.empty_cache()
    return out


def optimizer_study(local, seeds=(11, 12, 13, 14, 15, 16), frames=300, n_envs=1024):
    """Tracking error (median ADD of the argmin estimate over seeded
    trajectories, mm) and window time of each optimizer of Sec. III-D at the
    same N: the elite-weighted Gaussian resample, WRS, REPS, and REPS with
    exploration by velocity kicks instead of pose noise; and the paper's two
    baselines (Sec. IV): EYE (the same N noisy samples, no updates) and OLP
    (one simulation from the nominal pose)."""
    import dataclasses
    import torch
    from paper_2002_12160_gb300 import tracking, workloads as W
    torch.cuda.set_device(local)
    variants = {"elite": {"kind": "elite"}, "wrs": {"kind": "wrs"}, "reps": {"kind": "reps"},
                "reps_velocity": {"kind": "reps", "explore": "velocity"},
                "eye": {"baseline": "eye"}, "olp": {"baseline": "olp"}}
    out = {}
    for name in ["tracking_cyl64", "tracking_box27"]:
        res = {}
        for label, kw in variants.items():
            kw = dict(kw)
            baseline = kw.pop("baseline", None)
            n = 1 if baseline == "olp" else n_envs
            adds, times = [], []
            for seed in seeds:
                wl = W.make_workload(name, n_envs=n, frames=frames, seed=seed)
                wl.opt = dataclasses.replace(wl.opt, **kw)
                tr = tracking.Tracker(wl, n_envs=n)
                tr.prepare()
                if baseline == "olp":
                    tr.prepare_open_loop()
                step = tr.window_eye if baseline else tr.window
                nw = frames // tr.T
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                step(0)   # capture
                torch.cuda.synchronize()
                e0.record()
                for w in range(1, nw):
                    step(w)
                e1.record()
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1) / (nw - 1))
                adds.append(tr.add_mm(nw * tr.T))
                tr.close()
            res[label] = {"add_mm_median": statistics.median(adds), "add_mm_mean": float(np.mean(adds)),
                          "ms_per_window": statistics.median(times), "add_mm": adds}
        out[name] = res
    torch.cuda.empty_cache()
    return {"n_envs": n_envs, "frames": frames, "seeds": list(seeds), **out}


def warm_study(local, seeds=(11, 12, 13, 14, 15, 16), frames=300, n_envs=1024, n_conv=256, hold_at=40,
               hold_frames=90):
    """The warm-started solver (each contact starts from its (link, sphere)
    pair's final impulse of the previous substep):
    - convergence at a fixed iteration count I, in a held grasp (the command
      frozen at frame `hold_at` for `hold_frames` frames, n_conv sampled
      cylinder states): the object's residual speed (creep of an unconverged
      solve) and its distance from where a 200-iteration solve holds it;
    - tracking (median ADD over seeded trajectories, mm) and window time with
      the elite optimizer at I = 5, 10 and 20, warm and cold, against a ground
      truth simulated with a converged (200-iteration) solve."""
    import dataclasses
    import torch
    from paper_2002_12160_gb300 import inhand, tracking, workloads as W
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    conv = {}
    nf = hold_at + hold_frames
    wl = W.make_workload("tracking_cyl64", n_envs=n_conv, frames=nf)
    qh = wl.q_traj[:nf + 1].copy()
    qh[hold_at:] = qh[hold_at]
    q = torch.from_numpy(qh).contiguous().to(dev)

    def held(iters, warm):
        w2 = dataclasses.replace(wl, sim=dataclasses.replace(wl.sim, iters=iters, warm_start=warm))
        sim = inhand.make_sim(w2, n_envs=n_conv, max_frames=nf)
        sim.sim_set_commands(0, q)
        sim.sim_sample_initial(wl.nominal_pose, wl.init.sigma_p, wl.init.sigma_r, wl.init.m_range, wl.init.mu_range)
        sim.sim_step(0, nf)
        pose, vel, _, status = (t.double() for t in sim.sim_get_state())
        sim.close()
        return pose[:, :3], vel[:, :3].norm(dim=1), status

    x_ref, _, st_ref = held(200, False)
    for iters in (2, 5, 10, 20):
        row = {}
        for mode in ("cold", "warm"):
            x, speed, st = held(iters, mode == "warm")
            ok = (st == 0) & (st_ref == 0)
            row[mode] = {"creep_mm_per_s": 1e3 * speed[ok].mean().item(),
                         "offset_mm": 1e3 * (x - x_ref)[ok].norm(dim=1).median().item(),
                         "envs": int(ok.sum().item())}
        conv[str(iters)] = row
    track = {}
    for name in ["tracking_cyl64", "tracking_box27"]:
        res = {}
        for iters in (5, 10, 20):
            for warm in (False, True):
                adds, times = [], []
                for seed in seeds:
                    wl_t = W.make_workload(name, n_envs=n_envs, frames=frames, seed=seed)
                    gt_sim = dataclasses.replace(wl_t.sim, iters=200)
                    wl_t.sim = dataclasses.replace(wl_t.sim, iters=iters, warm_start=warm)
                    wl_t.iters[:] = iters
                    tr = tracking.Tracker(wl_t, n_envs=n_envs, gt_sim=gt_sim)
                    tr.prepare()
                    nw = frames // tr.T
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    tr.window(0)
                    torch.cuda.synchronize()
                    e0.record()
                    for w in range(1, nw):
                        tr.window(w)
                    e1.record()
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1) / (nw - 1))
                    adds.append(tr.add_mm(nw * tr.T))
                    tr.close()
                res[f"{'warm' if warm else 'cold'}_i{iters}"] = {
                    "add_mm_median": statistics.median(adds), "ms_per_window": statistics.median(times),
                    "add_mm": adds}
        track[name] = res
    torch.cuda.empty_cache()
    return {"convergence": {"what": f"held grasp (command frozen at frame {hold_at} for {hold_frames} frames), "
                                    f"{n_conv} sampled cylinder states: mean object speed and median offset "
                                    "from a 200-iteration solve", "by_iters": conv},
            "tracking": {"n_envs": n_envs, "frames": frames, "seeds": list(seeds),
                         "ground_truth": "200-iteration cold solve", **track}}


# Work model of the PD-hand step kernel (step_pd.cu), counted from its source
# the same way (FMA = 2, a sincos = 20): per env-substep the fingers'
# kinematics (570 per finger: quaternion chain, link axes, joint axes), the PD
# prediction (9 per joint), link culling (25 per link) and the object's
# prediction and inertia (145); per cluster test 25 (centre to world and the
# reach test); per pair tested 30; per contact the set-up with
# its joints' share (140) and the pad and slip sums (45); per contact-iteration
# the update against the link twist and the per-link sums (103); per
# env-iteration the joint updates (36 per joint) and the links' twists from
# them (24 per joint: each joint's contribution and a 4-lane prefix).
def pd_flops(work, scene, spheres):
    F, D, Lk = scene.n_fingers, scene.n_joints, scene.n_links
    per_substep = 570 * F + 9 * D + 25 * Lk + 145 + 15 * spheres
    return (work["env_substeps"] * per_substep + work["cluster_tests"] * 25 + work["pairs"] * 30 + work["contacts"] * 185 +
            work["contact_iters"] * 103 + work["env_iters"] * (60 * D + 30))


def pd_study(local, seeds=(11, 12, 13, 14, 15, 16), frames=300, n_envs=1024, windows=5, budget_s=10.0,
             speed_only=False, peak_tf=None):
    """The PD-driven hand (joints as state, full observation, full cost):
    - throughput on the cylinder trajectory at N = n_envs and 8 n_envs: per
      window one T-frame PD step launch, then the full cost of every frame
      (two launches), the per-frame argmin and the optimizer, timed with CUDA
      events (L2 flushed before every window), the step call (the step launch
      and its cost launches) separately with its counted work against the
      FP32 peak; and the same window as per-frame step and full-cost
      launches;
    - the oracle's PD step on the host, single thread, on a bounded sample;
    - tracking error (median ADD over seeded trajectories, mm) with the full
      cost, without the slip terms, and with the force and contact terms only
      (the paper's ablation of contact and slip feedback), ground truth and
      trackers all with the PD hand."""
    import dataclasses
    import torch
    import oracle as O
    from paper_2002_12160_gb300 import tracking, workloads as W
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    if peak_tf is None:
        peak_tf = measure_fp32_peak(local)["tflops"]

    def throughput_at(n):
        wl = W.make_workload("tracking_cyl64", n_envs=n, frames=frames, seed=seeds[0])
        wl.sim = dataclasses.replace(wl.sim, hand="pd")
        tr = tracking.Tracker(wl, n_envs=n)
        tr.prepare()
        T = tr.T
        for w in range(2):   # warm-up windows
            tr.window_pd(w)
        torch.cuda.synchronize()
        tr.sim.sim_work_counters(reset=True)
        win_ms, step_ms = [], []
        st_stream = torch.cuda.current_stream()
        for w in range(2, 2 + windows):   # the window: one T-frame step launch, argmin, optimizer
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            f0 = w * T
            ev[0].record(st_stream)
            tr.sim.sim_step_frames_full(f0, tr.obs_q[f0:f0 + T], tr.obs_pp[f0:f0 + T], tr.obs[f0:f0 + T],
                                        tr.obs_slip[f0:f0 + T])
            ev[1].record(st_stream)
            tr.sim.sim_frames_argmin(tr.est[f0:f0 + T], tr.argmin[f0:f0 + T])
            tr.sim.optimizer_update(wl.opt, w)
            ev[2].record(st_stream)
            torch.cuda.synchronize()
            win_ms.append(ev[0].elapsed_time(ev[2]))
            step_ms.append(ev[0].elapsed_time(ev[1]))
        work = tr.sim.sim_work_counters()
        unfused = []
        for w in range(2 + windows, 2 + 2 * windows):   # the same window as per-frame launches
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st_stream)
            tr.window_pd_unfused(w)
            e1.record(st_stream)
            torch.cuda.synchronize()
            unfused.append(e0.elapsed_time(e1))
        tr.close()
        n_launch = windows
        flop = pd_flops(work, wl.scene, max(len(x) for x in wl.scene.shapes)) / n_launch
        ms_win, ms_step = statistics.median(win_ms), statistics.median(step_ms)
        peak = peak_tf
        achieved = flop / (ms_step / 1e3) / 1e12
        return T, {"n_envs": n, "env_steps_per_s": n * T / (ms_win / 1e3), "ms_per_window": ms_win,
                   "step_kernel_ms_per_launch": ms_step, "frames_per_launch": T,
                   "tracking_frames_per_s": T / (ms_win / 1e3),
                   "unfused_ms_per_window": statistics.median(unfused),
                   "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                "frac": achieved / peak, "flop_per_launch": flop,
                                "peak_note": "measured FP32 FMA throughput (ih_fp32_peak)"},
                   "work_per_launch": {k: v / n_launch for k, v in work.items()}}

    T, throughput = throughput_at(n_envs)
    _, throughput_large = throughput_at(8 * n_envs)
    if speed_only:
        del flush
        return {"throughput": throughput, "throughput_large_n": throughput_large}
    # the oracle's PD step, bounded sample
    n_s = 16
    wl_s = W.make_workload("tracking_cyl64", n_envs=n_s, frames=frames, seed=seeds[0])
    sim_s = dataclasses.replace(wl_s.sim, hand="pd")
    osc = O.OracleScene(wl_s.scene)
    pose, theta = O.sample_initial(n_s, O.pose8_to7(wl_s.nominal_pose), wl_s.init, wl_s.seed)
    st = O.State(pose, np.zeros((n_s, 6)), theta).hand(wl_s.q_traj[0])
    t0, done = time.perf_counter(), 0
    while time.perf_counter() - t0 < budget_s and done < frames:
        O.step_pd(osc, sim_s, st, wl_s.q_traj, done, 1)
        done += 1
    el = time.perf_counter() - t0
    cpu = {"value": n_s * done / el, "unit": "env-steps/s", "cores": 1, "kind": "oracle",
           "sample": f"{n_s} envs x {done} frames of the cylinder trajectory with the PD hand, single thread, {el:.1f} s"}
    # tracking error by cost terms
    variants = {"full": None, "no_slip": (6, 7, 8, 9), "force_and_contact": (0, 1, 2, 6, 7, 8, 9)}
    track = {}
    for name in ["tracking_cyl64", "tracking_box27"]:
        res = {}
        for label, zero in variants.items():
            adds = []
            for seed in seeds:
                wl_t = W.make_workload(name, n_envs=n_envs, frames=frames, seed=seed)
                w_full = list(W.SimConfig().w_full)
                for k in (zero or ()):
                    w_full[k] = 0.0
                wl_t.sim = dataclasses.replace(wl_t.sim, hand="pd", w_full=tuple(w_full))
                tr = tracking.Tracker(wl_t, n_envs=n_envs)
                tr.prepare()
                nw = frames // tr.T
                for w in range(nw):
                    tr.window_pd(w)
                torch.cuda.synchronize()
                adds.append(tr.add_mm(nw * tr.T))
                tr.close()
            res[label] = {"add_mm_median": statistics.median(adds), "add_mm": adds}
        track[name] = res
    del flush
    torch.cuda.empty_cache()
    return {"workload": f"tracking_cyl64 with the PD hand, N = {n_envs}, windows of {T} frames",
            "throughput": throughput, "throughput_large_n": throughput_large, "cpu_baseline": cpu,
            "tracking": {"n_envs": n_envs, "frames": frames, "seeds": list(seeds), **track}}


def flops_of(work, wl):
    S = max(len(x) for x in wl.scene.shapes)
    per_substep = (FLOP_PER_ENV_SUBSTEP + FLOP_PER_LINK * wl.scene.n_links + FLOP_PER_CLUSTER * ((S + 7) // 8) +
                   FLOP_PER_SPHERE * S)
    return (work["env_substeps"] * per_substep + work["pairs"] * FLOP_PER_PAIR +
            work["cluster_tests"] * FLOP_PER_CLUSTER_TEST + work["contacts"] * FLOP_PER_CONTACT +
            work["contact_iters"] * FLOP_PER_CONTACT_ITER + work["env_iters"] * FLOP_PER_ENV_ITER)


def measure_fp32_peak(local):
    """FP32 FMA throughput of this GPU (ih_fp32_peak), with the SM clock sampled
    while it runs: the denominator of the step kernels' ALU roofline."""
    import torch
    from paper_2002_12160_gb300 import inhand
    torch.cuda.set_device(local)
    inhand.fp32_peak(iters=256, reps=2)   # warm-up
    with ClockSampler(local) as clk:
        tf, ms, sms = inhand.fp32_peak(iters=2048, reps=60)
    return {"tflops": tf, "ms_per_launch": ms, "sms": sms, "clocks": clk.summary(),
            "what": "FMA-chain kernel (8 independent chains per thread, 2048 threads per SM), "
                    "FMA = 2 flop, CUDA events over 60 launches"}


def summarize(m, peak_tf, hbm_gbs, world=1):
    """Throughput and roofline of one measured workload point: the window's
    env-steps/s and tracking frames/s; the step kernel's counted flops and
    algorithmic bytes per window-mode launch against its own CUDA-event time."""
    wl, n, T, ms = m["wl"], m["n"], m["T"], m["ms"]
    out = {"n_envs": n, "ms_per_window": ms, "env_steps_per_s": world * n * T / (ms / 1e3),
           "tracking_frames_per_s": T / (ms / 1e3),
           "step_shape": {"threads_per_env": m["chosen"][0], "contacts_per_thread": m["chosen"][1],
                          "autotune_ms": {f"{a}x{b}": round(v, 4) for (a, b), v in m["tune_ms"].items()}}}
    if "step_ms" in m:
        step_ms = m["step_ms"]
        flop = flops_of(m["work_t"], wl) / m["step_launches"]
        # one window-mode launch: state in/out once, the last frame's forces, the
        # window sum, and every frame's window mean (8 B) and pose (32 B)
        step_bytes = n * STATE_BYTES_PER_ENV + n * wl.scene.n_pads * 12 + n * 16 + T * n * 40
        out.update({"step_kernel_ms": step_ms, "flop_per_launch": flop,
                    "fp32": {"achieved_tflops": flop / (step_ms / 1e3) / 1e12,
                             "frac": flop / (step_ms / 1e3) / 1e12 / peak_tf},
                    "hbm": {"bytes_per_launch": step_bytes, "achieved_gbs": step_bytes / (step_ms / 1e3) / 1e9,
                            "frac": step_bytes / (step_ms / 1e3) / 1e9 / hbm_gbs},
                    "work_per_env_frame": {k: v / (m["step_launches"] * T * n) for k, v in m["work_t"].items()}})
    if "adjoint" in m:
        out["forward_adjoint"] = m["adjoint"]
    return out


def largest_n_at_30hz(workload, local, shape, rate_hint, floor_n, peak_tf, hbm_gbs, step=4096, max_points=5):
    """Bounded search for the largest N whose tracking window holds >= 30
    tracking frames/s: each point predicts the boundary from its own measured
    throughput (N = rate / 30 on a grid of `step` environments; one step
    further when the prediction is the point itself), until the boundary is
    bracketed within one grid step or `max_points` points are spent; each
    point also times the step kernel alone (its FP32 and HBM roofline)."""
    import torch
    pts = []

    def point(n):
        r = measure(workload, n, 3, 2, shape, 0, 1, local, n_timing=2)
        p = summarize(r, peak_tf, hbm_gbs)
        p.pop("work_per_env_frame", None)
        pts.append(p)
        torch.cuda.empty_cache()
        return p["tracking_frames_per_s"], p["env_steps_per_s"]

    lo, hi = floor_n, None     # floor_n holds 30 Hz (measured in the sweep)
    n = max(lo + step, step * int(rate_hint / 30.0 // step))
    while len(pts) < max_points:
        f, rate = point(n)
        if f >= 30.0:
            lo = max(lo, n)
        else:
            hi = n if hi is None else min(hi, n)
        if hi is not None and hi - lo <= step:
            break
        pred = step * int(rate / 30.0 // step)
        if hi is None:
            n = max(lo + step, pred)
        elif lo <= floor_n:
            n = max(floor_n + step, min(hi - step, pred))
        else:
            n = lo + step * max(1, (hi - lo) // (2 * step))
    return {"largest_n_measured_at_30hz": lo, "smallest_n_measured_below_30hz": hi, "grid": step,
            "points": pts, "step_shape": list(shape) if shape else None}


def run_ours(args, rank, world, local):
    hbm_gbs, hbm_note = hbm_peak()
    peak = measure_fp32_peak(local)
    peak_tf = peak["tflops"]
    m = measure(args.workload, args.n_envs, args.steps, args.warmup, args.shape, rank, world, local,
                n_timing=3, n_e2e=40)
    main_pt = summarize(m, peak_tf, hbm_gbs, world)
    wl, n, T, ms = m["wl"], m["n"], m["T"], m["ms"]
    value = main_pt["env_steps_per_s"]
    clocks = m["clocks"]
    chosen, tune_ms = m["chosen"], m["tune_ms"]
    e2e = m["e2e"]
    e2e_line = {k: e2e[k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step")}
    e2e_line["value"] *= world
    e2e_line.update({"ms_per_step": e2e["ms_per_step"], "windows": e2e["windows"], "pipelined": True,
                     "host_waits_each_window": e2e["host_waits_each_window"]})
    line = {"metric": "env-steps/s", "value": value, "unit": "env-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "n_envs": n, "window_frames": T,
                       "spheres": sorted(set(int(len(x)) for x in wl.scene.shapes)), "links": wl.scene.n_links,
                       "pads": wl.scene.n_pads, "iters": sorted(set(int(i) for i in wl.iters[:n])),
                       "substeps": wl.sim.substeps,
                       "l2": "flushed (256 MB write) before every timed step", "parallelism": f"replicas{world}",
                       "step_shape": {"threads_per_env": chosen[0], "contacts_per_thread": chosen[1],
                                      "autotune_ms": {f"{a}x{b}": round(v, 4) for (a, b), v in tune_ms.items()}}},
            "tracking_frames_per_s": main_pt["tracking_frames_per_s"],
            "roofline": {"bound": "alu", "achieved": main_pt["fp32"]["achieved_tflops"], "peak": peak_tf,
                         "unit": "TFLOP/s", "frac": main_pt["fp32"]["frac"], "traffic": step_traffic(),
                         "traffic_unit": "bytes per launch",
                         "kernel": "step_kernel in window mode (one launch = the window's T scored frames)",
                         "step_kernel_ms": main_pt["step_kernel_ms"], "flop_per_launch": main_pt["flop_per_launch"],
                         "peak_note": f"measured FP32 FMA throughput of this GPU ({peak['sms']} SMs, "
                                      f"SM clock median {peak['clocks'].get('sm_mhz')} MHz during the probe)"},
            "hbm": {"step_bytes_per_launch": main_pt["hbm"]["bytes_per_launch"],
                    "achieved_gbs": main_pt["hbm"]["achieved_gbs"], "peak_gbs": hbm_gbs,
                    "frac": main_pt["hbm"]["frac"], "peak_note": hbm_note},
            "fp32_peak": peak,
            "work_per_env_frame": main_pt["work_per_env_frame"],
            "clocks": clocks,
            "gpu_launches": args.steps * 7,   # descriptor, T-frame step, per-frame argmin, 4 optimizer kernels
            "e2e": e2e_line,
            "add_mm_argmin_env": m["add_mm"]}
    if args.sweep:
        sweep = []
        for nn in [int(v) for v in args.sweep.split(",")]:
            r = measure(args.workload, nn, 3, 2, args.shape, rank, world, local, n_timing=0)
            fps = r["T"] / (r["ms"] / 1e3)
            sweep.append({"n_envs": nn, "ms_per_window": r["ms"], "tracking_frames_per_s": fps,
                          "env_steps_per_s": nn * fps, "step_shape": list(r["chosen"])})
        line["sweep"] = sweep
        ok = [x for x in sweep if x["tracking_frames_per_s"] >= 30.0]
        line["largest_n_measured_at_30hz"] = max((x["n_envs"] for x in ok), default=None)
    if world == 1 and not args.main_only:
        # config 2: the uneven batch in one launch per window, autotuned shape
        line["uneven_mixed"] = summarize(measure("uneven_mixed", 8192, 5, 3, None, 0, 1, local, n_timing=2),
                                         peak_tf, hbm_gbs)
        # config 4: the mug sweep, forward-only and forward + adjoint (one 10-frame window's horizon)
        sweep = []
        for nn in (1024, 4096, 16384, 32768):
            sweep.append(summarize(measure("sweep_mug128", nn, 5, 3, None, 0, 1, local, n_timing=2,
                                           adjoint_h=10), peak_tf, hbm_gbs))
        line["sweep_mug128"] = {"what": "mug of 128 spheres, 5 fingers, 16 pads, I = 40, 4 substeps; forward = the "
                                        "tracking window; forward_adjoint = sim_adjoint of a 10-frame horizon on "
                                        "every environment", "points": sweep}
        sat = sweep[-1]
        shp = (sat["step_shape"]["threads_per_env"], sat["step_shape"]["contacts_per_thread"])
        ok = [p["n_envs"] for p in sweep if p["tracking_frames_per_s"] >= 30.0]
        line["sweep_mug128"]["largest_n_at_30hz"] = largest_n_at_30hz(
            "sweep_mug128", local, shp, sat["env_steps_per_s"], max(ok) if ok else 1024, peak_tf, hbm_gbs)
        # config 3: forward + adjoint of a 30-frame horizon, N = 1024, box and cylinder
        line["adjoint"] = {"what": "forward + reverse-mode gradient of the horizon cost (sim_adjoint), "
                                   "every environment, H = 30 frames, checkpoints every 10",
                           "forward_env_steps_per_s": value / world, **measure_adjoint(local)}
        line["pd_hand"] = pd_study(local, speed_only=True, peak_tf=peak_tf)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload)
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    parts = {"adjoint": lambda: {"adjoint": measure_adjoint(local)},
             "optimizers": lambda: {"optimizers": optimizer_study(local)},
             "pd": lambda: {"pd_hand": pd_study(local)},
             "pd_speed": lambda: {"pd_hand": pd_study(local, speed_only=True)},
             "warm": lambda: {"warm_start": warm_study(local)},
             "refine": lambda: {"refinement": refine_study(local)}}
    if args.part in parts:
        if rank == 0:
            print(json.dumps({"part": args.part, **parts[args.part]()}), flush=True)
        return
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_ours(args, rank, world, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
