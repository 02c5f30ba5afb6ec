"""Benchmark of the batched, graph-captured FP64 RK4 level step.

Default workload: one periodic 256^3 box, variable c2 (8 seeded bumps),
Gaussian pulse, dt = 0.25 h; one benchmark step = 100 RK4 steps (the
headline single-box workload).  Metric: grid-point RK4 updates per second
(interior points x RK4 steps / s).  Prints ONE JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the
workload on its own GPU (no data-path collective); timing is the maximum
over ranks and `value` counts the updates of all ranks (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FP64 grid-point RK4 updates/s"
# the headline workload, named the same in both arms
WORKLOAD = "periodic box 256^3, variable c2 (8 seeded bumps), Gaussian pulse, RK4 dt=0.25h"
UNIT = "updates/s"
RK4_STEPS_PER_BENCH_STEP = 100
N_EDGE = 256
# algorithmic bytes per interior point per RK4 step of the nested stage form:
# stage 1 reads y.u (stencil), y.pi, c2 and writes w.u, w.pi (5 doubles);
# stages 2-4 read w.u (stencil), w.pi, y.u, y.pi, c2 and write 2 (7 doubles)
BYTES_PER_POINT_STEP = 8 * (5 + 7 + 7 + 7)
BYTES_PER_POINT_STAGE = BYTES_PER_POINT_STEP / 4
# two stages per pass: pass A reads y.u, y.pi (stencils), q, q/3 and writes
# w_2.u, w_2.pi, L y.u (7 doubles); pass B reads w_2.u, w_2.pi (stencils),
# y.u, y.pi, q, L y.u and writes y.u, y.pi (8 doubles)
BYTES_PER_POINT_PASS = {"A": 8 * 7, "B": 8 * 8}
# FP64 pipe instructions per point per stage (FP64 form): 10 adds + 2 FMAs
# for the sum, 1 multiply by c2, 2 update FMAs; fixed form: the conversion
# of the sum and 2 update FMAs (the pass kernels convert on the integer pipes
# and need 4 FMAs per pass, i.e. 2 per stage)
FP64_OPS_PER_POINT_STAGE = {"fp64": 15, "fixed": 3}
FP64_OPS_PER_POINT_PASS = {"fp64": 28, "fixed": 4}
# FP64 FMA rate of this GPU (G FMA/s), measured with a probe kernel of
# back-to-back independent DFMAs timed by CUDA events: about 2 lanes per
# clock per SM at 2.07 GHz
FP64_FMA_RATE_G = 597.0
# bytes per point and RK4 step of the classic unfused stage form (each of
# the 3-register stage arrays streamed once per stage): 38 doubles
BYTES_PER_POINT_STEP_CLASSIC = 304
# seconds of CPU work the oracle's cpu_baseline sample aims at
CPU_SAMPLE_S = 12.0
# RK4 steps of the oracle per step of the reference arm
REF_RK4_STEPS = 10
# what the line's dtype means in each arithmetic form of the Laplacian sum
DTYPE_LABEL = {
    "fixed": "f64 (fixed-point Laplacian sum: each input truncated to 2^-54 of its "
             "field's domain maximum, the sum exact in int64 and rounded once; RK "
             "updates in FP64)",
    "fp64": "f64",
}
# run-time tuning results (tile per box-size class) are cached here between runs
TUNE_CACHE = os.path.join(ROOT, "paper_1308_1343_gb300", "_build", "tune_cache.txt")


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--arith", choices=["fixed", "fp64"], default="fixed")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the uneven-level, ensemble, two-level and adjoint measurements")
    p.add_argument("--extras", default=",".join(EXTRAS),
                   help="comma-separated subset of %s to measure" % ",".join(EXTRAS))
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    return p.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(t: float, dist=None, device=None) -> float:
    """The largest of every rank's value (the job's time); t itself when
    running alone."""
    if dist is None:
        return t
    import torch
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_rate(units_per_rank: float, t_max: float, world: int) -> float:
    """Whole-job throughput: every rank processes units_per_rank units (an
    independent replica) and the job takes the slowest rank's time."""
    return units_per_rank * world / t_max


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.rows = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", gpu_id, "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 8:
                self.rows.append(parts)

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = []
        mx = None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
            except ValueError:
                continue
            for n, v in zip(names, r[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _kernel_source_hash():
    h = hashlib.sha256()
    for f in ("kernels.cu", "kernels.cuh", "kernels_ws.cuh", "descriptors.hpp", "launch.hpp"):
        with open(os.path.join(ROOT, "paper_1308_1343_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _stencil_roofline(lev, B, npts):
    """Algorithmic GB/s of the level's stencil kernels in its current form,
    from the per-launch CUDA events of the last SC_MODE_TIMED call:
    (achieved GB/s, mean launch ms, mean bytes per launch, launches, name)."""
    if lev.get_fusion() == 2:
        name = "pair_ws_kernel" if lev.get_pass_kernel() == B.SC_PASS_WARP_SPECIALISED \
            else "pair_kernel"
        ta, na = lev.kernel_time(B.SC_KERNEL_PAIR_A)
        tb, nb = lev.kernel_time(B.SC_KERNEL_PAIR_B)
        if not (na and nb):
            return None, None, None, 0, name
        nbytes = (BYTES_PER_POINT_PASS["A"] * na + BYTES_PER_POINT_PASS["B"] * nb) * npts
        return (nbytes / ((ta + tb) * 1e-3) / 1e9, (ta + tb) / (na + nb), nbytes / (na + nb),
                na + nb, name + " (passes A and B)")
    sm, sl, _, _ = lev.kernel_times()
    if not sl:
        return None, None, None, 0, "fwd_stage_kernel"
    return (BYTES_PER_POINT_STAGE * npts * sl / (sm * 1e-3) / 1e9, sm / sl,
            BYTES_PER_POINT_STAGE * npts, sl, "fwd_stage_kernel")


def _traffic(kernel_hash, workload):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, or None if it was taken on another version of the kernel."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        for line in open(path):
            kv = dict(x.split("=", 1) for x in line.split() if "=" in x)
            if kv.get("kernel") == kernel_hash and kv.get("workload") == workload:
                return float(kv["bytes_per_launch"])
    except OSError:
        pass
    return None


# ----------------------------------------------------------------------------
# the CPU oracle (reference arm and cpu_baseline)
# ----------------------------------------------------------------------------

def _oracle_rate(inst, nsteps):
    from oracle import oracle
    cores = len(os.sched_getaffinity(0))
    used = oracle.set_threads(cores)
    t0 = time.perf_counter()
    oracle.rk4_periodic(inst.u, inst.pi, inst.c2, inst.dom.h, inst.dt, nsteps)
    dt = time.perf_counter() - t0
    oracle.set_threads(1)
    n = inst.u.size
    return n * nsteps / dt, used, dt


def run_reference(a, ws, rank):
    if rank != 0:
        return
    from paper_1308_1343_gb300 import workloads as W
    inst = W.single_box(N_EDGE, seed=2)
    for _ in range(a.warmup):
        _oracle_rate(inst, 1)
    rates, times = [], []
    used = 1
    for _ in range(a.steps):
        r, used, dt = _oracle_rate(inst, REF_RK4_STEPS)
        rates.append(r)
        times.append(dt)
    total_t = sum(times)
    value = inst.u.size * REF_RK4_STEPS * len(times) / total_t
    sample = "%d RK4 steps of the 256^3 workload per benchmark step" % REF_RK4_STEPS
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * total_t / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "points": inst.u.size,
                   "rk4_steps_per_step": REF_RK4_STEPS,
                   "workload_rk4_steps_per_step": RK4_STEPS_PER_BENCH_STEP,
                   "rk4_steps_note": "the oracle advances %d of the workload's %d RK4 steps "
                                     "per benchmark step, a bounded sample that keeps the "
                                     "run within minutes; the metric counts updates per "
                                     "second, so the two arms' rates compare"
                                     % (REF_RK4_STEPS, RK4_STEPS_PER_BENCH_STEP),
                   "arith": "fp64 (oracle)", "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def _time_steps(torch, lev, u, pi, c2, dt, nsteps, mode, reps, stream):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        lev.rk4_step(u, pi, c2, dt, nsteps, mode, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    lev.sync(stream)
    return e0.elapsed_time(e1) / 1e3


EXTRAS = ("fp64", "uneven", "ensemble", "two_level", "adjoint", "dist")


def _time_grad(torch, lev, u0, pi0, c2, dt, nsteps, ckpt, stream, reps=2):
    """Wall time of a taped forward and of the backward of the misfit of u_T
    against u0 (the second of `reps` repetitions)."""
    uT = torch.empty_like(u0)
    seed = torch.empty_like(u0)
    g = [torch.empty_like(u0) for _ in range(3)]
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lev.forward_tape(u0, pi0, c2, dt, nsteps, ckpt, uT, None, stream=stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        lev.misfit(uT, u0, seed, stream=stream)
        lev.backward_tape(c2, seed, None, g[0], g[1], g[2], stream=stream)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
    lev.sync(stream)
    return t1 - t0, t2 - t1


def _extras(torch, W, B, Level, arith, stream, which=EXTRAS):
    out = {}
    if "fp64" in which and arith == B.SC_ARITH_FIXED:
        out["fp64_arith"] = _fp64_rate(torch, W, B, Level, stream)
    if "uneven" in which:
        out["uneven_level"] = _uneven(torch, W, B, Level, arith, stream)
    if "ensemble" in which:
        out["ensemble"] = _ensemble(torch, W, B, Level, arith, stream)
    if "two_level" in which:
        # two-level hierarchy: coarse 256^3 periodic, fine region 256^3 points
        # (the central eighth of the domain at half the spacing), 20 steps
        out["two_level"] = _two_level(torch, W, B, Level, arith, stream)
    if "adjoint" in which:
        out["adjoint"] = _adjoint(torch, W, B, Level, arith, stream)
    if "dist" in which:
        out["dist_emulated"] = _dist_emulated(torch, W, B, Level, arith, stream)
    return out


def _dist_emulated(torch, W, B, Level, arith, stream):
    """The distributed level's kernels on one GPU: the 64-box level split over
    two ranks (spatial bisection), both ranks' parts in this process, their
    exchange blocks copied device to device between the passes (no NCCL, no
    second GPU): what the partition, the pack and unpack kernels and the split
    step cost against the one-level graph run of the same level."""
    from paper_1308_1343_gb300.dist import DistLevel, partition, step_ranks
    inst = W.uneven_level()
    boxes = [(lo, hi, 0) for lo, hi in inst.boxes]
    doms = [dict(hi=inst.dom.n, h=inst.dom.h, periodic=7)]
    nranks = 2
    owner = partition(boxes, nranks, B.SC_DIST_BISECT)
    levs = [DistLevel(boxes, doms, nranks, r, owner) for r in range(nranks)]
    for L in levs:
        L.set_arith(arith)
    us = [L.to_device([inst.u]) for L in levs]
    ps = [L.to_device([inst.pi]) for L in levs]
    cs = [L.to_device([inst.c2], fill=1.0) for L in levs]
    step_ranks(levs, us, ps, cs, inst.dt, 2, stream=stream)
    torch.cuda.synchronize()
    nsteps = 10
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    step_ranks(levs, us, ps, cs, inst.dt, nsteps, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    for L in levs:
        L.sync(stream)
    t = e0.elapsed_time(e1) / 1e3
    sent = sum(L.send_doubles for L in levs) * 8 * 2  # two exchanges per step
    out = {"workload": "512x512x256 periodic domain, 64 bisected boxes, over 2 ranks "
                       "(spatial bisection) held in one process on one GPU; exchange blocks "
                       "copied device to device between the passes (no NCCL)",
           "ranks": nranks, "boxes_per_rank": [len(L.boxes) for L in levs],
           "rk4_steps": nsteps, "updates_per_s": inst.u.size * nsteps / t,
           "ms_per_step": 1e3 * t / nsteps, "exchanged_bytes_per_step": sent}
    for L in levs:
        L.close()
    del us, ps, cs
    torch.cuda.empty_cache()
    return out


def _fp64_rate(torch, W, B, Level, stream):
    """The headline workload with FP64 adds and FMAs in the Laplacian sum
    (SC_ARITH_FP64) instead of the fixed-point sum: the cost of IEEE
    arithmetic throughout, same form choice, tuning and timing."""
    inst = W.single_box(N_EDGE, seed=2)
    lev = Level.from_instances([inst])
    lev.set_arith(B.SC_ARITH_FP64)
    lev.autotune(seed=2, budget_ms=2000.0, abort_factor=2.0, cache_path=TUNE_CACHE,
                 stream=stream)
    u, pi = lev.to_device([inst.u]), lev.to_device([inst.pi])
    c2 = lev.to_device([inst.c2], fill=1.0)
    nsub = RK4_STEPS_PER_BENCH_STEP
    _time_steps(torch, lev, u, pi, c2, inst.dt, nsub, B.SC_MODE_GRAPH, 3, stream)
    reps = 3
    t = _time_steps(torch, lev, u, pi, c2, inst.dt, nsub, B.SC_MODE_GRAPH, reps, stream)
    out = {"workload": WORKLOAD + ", FP64 Laplacian sums",
           "arith": "fp64", "dtype": DTYPE_LABEL["fp64"], "stages_per_pass": lev.get_fusion(),
           "updates_per_s": inst.u.size * nsub * reps / t,
           "ms_per_step": 1e3 * t / reps, "rk4_steps_per_step": nsub}
    del lev, u, pi, c2
    torch.cuda.empty_cache()
    return out


def _uneven(torch, W, B, Level, arith, stream):
    """Uneven 64-box level: batched graph vs per-box launches, 50 RK4 steps."""
    inst = W.uneven_level()
    lev = Level.from_instances([inst])
    lev.set_arith(arith)
    lev.autotune(seed=3, budget_ms=3000.0, abort_factor=2.0, cache_path=TUNE_CACHE,
                 stream=stream)
    u, pi = lev.to_device([inst.u]), lev.to_device([inst.pi])
    c2 = lev.to_device([inst.c2], fill=1.0)
    n = inst.u.size
    res = {}
    for name, mode in (("graph", B.SC_MODE_GRAPH), ("per_box", B.SC_MODE_PER_BOX)):
        _time_steps(torch, lev, u, pi, c2, inst.dt, 5, mode, 1, stream)
        t = _time_steps(torch, lev, u, pi, c2, inst.dt, 50, mode, 1, stream)
        res[name] = n * 50 / t
    lev.rk4_step(u, pi, c2, inst.dt, 10, B.SC_MODE_TIMED, stream=stream)
    gbs, _, _, _, kname = _stencil_roofline(lev, B, n)
    hbm = _peaks().get("hbm_gbs")
    # whole-step view of both forms: the stencil kernels' algorithmic bytes per
    # point and RK4 step (ghost copies not counted) times the step rate
    per_pt = (sum(BYTES_PER_POINT_PASS.values()) if lev.get_fusion() == 2
              else BYTES_PER_POINT_STEP)
    frac = (lambda g: g / hbm if (g and hbm) else None)
    out = {
        "workload": "512x512x256 periodic domain, 64 bisected boxes, 50 RK4 steps",
        "boxes": len(inst.boxes), "points": n, "stages_per_pass": lev.get_fusion(),
        "graph_updates_per_s": res["graph"], "per_box_updates_per_s": res["per_box"],
        "stencil_kernel": kname, "stencil_kernel_gbs": gbs,
        "stencil_kernel_frac_of_measured_hbm": frac(gbs),
        "bytes_per_point_step": per_pt,
        "step_frac_of_measured_hbm": {name: frac(per_pt * r / 1e9) for name, r in res.items()},
    }
    # the level's gradient: 50 steps, checkpoints every 10, misfit seed
    u0, pi0 = lev.to_device([inst.u]), lev.to_device([inst.pi])
    t_fwd = _time_steps(torch, lev, u, pi, c2, inst.dt, 50, B.SC_MODE_GRAPH, 1, stream)
    t_tape, t_bwd = _time_grad(torch, lev, u0, pi0, c2, inst.dt, 50, 10, stream)
    out["gradient"] = {"rk4_steps": 50, "ckpt_every": 10, "t_forward_s": t_fwd,
                       "t_forward_tape_s": t_tape, "t_backward_s": t_bwd,
                       "ratio_backward_over_forward": t_bwd / t_fwd,
                       "ratio_total_over_forward": (t_tape + t_bwd) / t_fwd}
    del lev, u, pi, c2, u0, pi0
    torch.cuda.empty_cache()
    return out


def _ensemble(torch, W, B, Level, arith, stream):
    """256 independent periodic cubes of edge 24..96, 100 RK4 steps."""
    insts = W.ensemble()
    lev = Level.from_instances(insts)
    lev.set_arith(arith)
    u = lev.to_device([i.u for i in insts])
    pi = lev.to_device([i.pi for i in insts])
    c2 = lev.to_device([i.c2 for i in insts], fill=1.0)
    dts = [i.dt for i in insts]
    n = sum(i.u.size for i in insts)
    lev.autotune(seed=5, budget_ms=3000.0, abort_factor=2.0, cache_path=TUNE_CACHE,
                 stream=stream)
    _time_steps(torch, lev, u, pi, c2, dts, 5, B.SC_MODE_GRAPH, 1, stream)
    t = _time_steps(torch, lev, u, pi, c2, dts, 100, B.SC_MODE_GRAPH, 1, stream)
    # 100 RK4 steps plus the adjoint gradient of every instance (one misfit
    # per instance, checkpoints every 20)
    u0 = lev.to_device([i.u for i in insts])
    pi0 = lev.to_device([i.pi for i in insts])
    t_tape, t_bwd = _time_grad(torch, lev, u0, pi0, c2, dts, 100, 20, stream)
    out = {"workload": "256 periodic cubes, edges 24..96, own c2 and pulse, "
                       "100 RK4 steps, autotuned tiles",
           "points": n, "stages_per_pass": lev.get_fusion(),
           "graph_updates_per_s": n * 100 / t,
           "gradient": {"rk4_steps": 100, "ckpt_every": 20, "t_forward_s": t,
                        "t_forward_tape_s": t_tape, "t_backward_s": t_bwd,
                        "ratio_backward_over_forward": t_bwd / t,
                        "ratio_total_over_forward": (t_tape + t_bwd) / t}}
    del lev, u, pi, c2, u0, pi0
    torch.cuda.empty_cache()
    return out


def _adjoint(torch, W, B, Level, arith, stream):
    """Adjoint / forward ratio on the 128^3, 200-step differentiation
    workload, and where the backward's device time goes."""
    inst = W.gradient_problem(128, 4)
    lev = Level.from_instances([inst])
    lev.set_arith(arith)
    lev.autotune(seed=4, budget_ms=2000.0, abort_factor=2.0, cache_path=TUNE_CACHE,
                 stream=stream)
    u0, pi0 = lev.to_device([inst.u]), lev.to_device([inst.pi])
    c2 = lev.to_device([inst.c2], fill=1.0)
    u = u0.clone()
    pi = pi0.clone()
    _time_steps(torch, lev, u, pi, c2, inst.dt, 20, B.SC_MODE_GRAPH, 1, stream)
    u.copy_(u0)
    pi.copy_(pi0)
    t_fwd = _time_steps(torch, lev, u, pi, c2, inst.dt, 200, B.SC_MODE_GRAPH, 1, stream)
    uT = torch.empty_like(u0)
    seed = torch.empty_like(u0)
    g = [torch.empty_like(u0) for _ in range(3)]
    for rep in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lev.forward_tape(u0, pi0, c2, inst.dt, 200, 20, uT, None, stream=stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        lev.misfit(uT, u0, seed, stream=stream)
        lev.backward_tape(c2, seed, None, g[0], g[1], g[2], stream=stream)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
    lev.sync(stream)
    # where the backward's device time goes (separate, event-timed pass)
    lev.set_profiling(True)
    lev.forward_tape(u0, pi0, c2, inst.dt, 200, 20, uT, None, stream=stream)
    lev.backward_tape(c2, seed, None, g[0], g[1], g[2], stream=stream)
    torch.cuda.synchronize()
    names = {B.SC_KERNEL_STAGE_RECORD: "stage_record", B.SC_KERNEL_PAIR_A: "pass_a",
             B.SC_KERNEL_PAIR_B: "pass_b", B.SC_KERNEL_GATHER: "gather",
             B.SC_KERNEL_ADJ_A: "adj_a", B.SC_KERNEL_ADJ_B: "adj_b", B.SC_KERNEL_ADJ_C: "adj_combine"}
    kern = {}
    for k, name in names.items():
        ms, n = lev.kernel_time(k)
        kern[name] = {"ms": ms, "launches": n}
    lev.set_profiling(False)
    return {"workload": "128^3 periodic box, 200 RK4 steps, checkpoints every 20",
            "stages_per_pass": lev.get_fusion(), "t_forward_s": t_fwd,
            "t_forward_tape_s": t1 - t0, "t_backward_s": t2 - t1,
            "ratio_backward_over_forward": (t2 - t1) / t_fwd,
            "ratio_total_over_forward": (t2 - t0) / t_fwd, "backward_kernels": kern}


def _two_level(torch, W, B, Level, arith, stream):
    """Berger-Oliger steps of a two-level hierarchy; updates count both levels
    (coarse points once, fine points twice per step)."""
    from paper_1308_1343_gb300.level import Hierarchy
    n = 256
    lo, hi = (n // 2,) * 3, (3 * n // 2,) * 3
    coarse, (fu_h, fp_h, fc_h) = W.refined_fields(n, 7, lo, hi)
    c = Level.from_instances([coarse])
    f = Level([(lo, hi, 0)], [dict(lo=lo, hi=hi, h=0.5 / n, periodic=0)])
    for lev in (c, f):
        lev.set_arith(arith)
        lev.autotune(seed=6, budget_ms=2000.0, abort_factor=2.0, cache_path=TUNE_CACHE,
                     stream=stream)
    h = Hierarchy(c, f)
    cu, cp = c.to_device([coarse.u]), c.to_device([coarse.pi])
    cc = c.to_device([coarse.c2], fill=1.0)
    fu, fp, fc = f.to_device([fu_h]), f.to_device([fp_h]), f.to_device([fc_h], fill=1.0)
    nsteps = 20
    h.step(cu, cp, cc, fu, fp, fc, coarse.dt, 2, stream=stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h.step(cu, cp, cc, fu, fp, fc, coarse.dt, nsteps, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    c.sync(stream)
    f.sync(stream)
    t = e0.elapsed_time(e1) / 1e3
    nc, nf = coarse.u.size, fu_h.size
    npro, nres = h.counts()
    # the levels alone, for the split of the time
    tc = _time_steps(torch, c, cu, cp, cc, coarse.dt, nsteps, B.SC_MODE_GRAPH, 1, stream)
    tf = 0.0
    for _ in range(2 * nsteps):
        tf += _time_steps(torch, f, fu, fp, fc, 0.5 * coarse.dt, 1, B.SC_MODE_GRAPH, 1, stream)
    h.close()
    return {"workload": "periodic 256^3 coarse level (h = 1/256) + fine region of 256^3 points "
                        "(h = 1/512, the central eighth), buffer 4, 20 Berger-Oliger steps",
            "coarse_points": nc, "fine_points": nf, "prolongated_points_per_fine_step": npro,
            "restricted_points_per_step": nres,
            "stages_per_pass": [c.get_fusion(), f.get_fusion()],
            "updates_per_s": (nc + 2 * nf) * nsteps / t, "ms_per_step": 1e3 * t / nsteps,
            "coarse_level_alone_ms_per_step": 1e3 * tc / nsteps,
            "fine_level_alone_ms_per_two_steps": 1e3 * tf / nsteps}


def run_ours(a, ws, rank, local):
    import torch
    from paper_1308_1343_gb300 import binding as B
    from paper_1308_1343_gb300 import build as BUILD
    from paper_1308_1343_gb300 import workloads as W
    from paper_1308_1343_gb300.level import Level

    torch.cuda.set_device(local)
    BUILD.build()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    arith = B.SC_ARITH_FIXED if a.arith == "fixed" else B.SC_ARITH_FP64
    stream = torch.cuda.current_stream()
    inst = W.single_box(N_EDGE, seed=2)
    npts = inst.u.size
    lev = Level.from_instances([inst])
    lev.set_arith(arith)
    lev.autotune(seed=2, budget_ms=2000.0, abort_factor=2.0, cache_path=TUNE_CACHE,
                 stream=stream)
    u0 = lev.to_device([inst.u])
    pi0 = lev.to_device([inst.pi])
    c2 = lev.to_device([inst.c2], fill=1.0)
    u, pi = u0.clone(), pi0.clone()
    nsub = RK4_STEPS_PER_BENCH_STEP

    for _ in range(a.warmup):
        lev.rk4_step(u, pi, c2, inst.dt, nsub, B.SC_MODE_GRAPH, stream=stream)
    lev.sync(stream)
    torch.cuda.synchronize()

    props = torch.cuda.get_device_properties(local)
    gpu_id = "GPU-" + str(getattr(props, "uuid", "")) if getattr(props, "uuid", None) else str(local)
    clocks = Clocks(gpu_id)
    launches0 = lev.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # an event between benchmark steps too: best and median step besides the total
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps + 1)]
    evs[0].record(stream)
    for k in range(a.steps):
        lev.rk4_step(u, pi, c2, inst.dt, nsub, B.SC_MODE_GRAPH, stream=stream)
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t = evs[0].elapsed_time(evs[-1]) / 1e3
    per_step = sorted(evs[k].elapsed_time(evs[k + 1]) for k in range(a.steps))
    clk = clocks.stop()
    lev.sync(stream)
    launches = lev.launch_count() - launches0
    t = max_over_ranks(t, dist, "cuda")
    value = job_rate(npts * nsub * a.steps, t, ws)

    # dominant kernels: the stencil kernels of the form the tuner chose,
    # timed per launch with CUDA events on the launching stream
    form = lev.get_fusion()
    lev.rk4_step(u, pi, c2, inst.dt, nsub, B.SC_MODE_TIMED, stream=stream)
    achieved, avg_ms, bytes_launch, nlaunch, kname = _stencil_roofline(lev, B, npts)
    gather_ms, gather_n = lev.kernel_time(B.SC_KERNEL_GATHER)
    lev.sync(stream)
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs")
    khash = _kernel_source_hash()
    traffic = _traffic(khash, "single256_f%d" % form)
    ops = (FP64_OPS_PER_POINT_PASS if form == 2 else FP64_OPS_PER_POINT_STAGE)[a.arith]
    fp64_achieved = 2 * ops * npts / (avg_ms * 1e-3) / 1e12  # FMA = 2 flops upper estimate

    # end to end through the C ABI with pinned host buffers
    hu = torch.from_numpy(lev.scatter([inst.u])).pin_memory()
    hp = torch.from_numpy(lev.scatter([inst.pi])).pin_memory()
    hc = torch.from_numpy(lev.scatter([inst.c2], fill=1.0)).pin_memory()
    ou = torch.empty_like(hu).pin_memory()
    op = torch.empty_like(hp).pin_memory()
    hun, hpn, hcn, oun, opn = (x.numpy() for x in (hu, hp, hc, ou, op))
    lev.rk4_step_host(hun, hpn, hcn, inst.dt, nsub, oun, opn, stream=stream)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        lev.rk4_step_host(hun, hpn, hcn, inst.dt, nsub, oun, opn, stream=stream)
    te2e = time.perf_counter() - t0
    te2e = max_over_ranks(te2e, dist, "cuda")
    fbytes = lev.field_size * 8
    e2e = {"value": job_rate(npts * nsub * a.steps, te2e, ws), "unit": UNIT,
           "h2d_bytes_per_step": 3 * fbytes, "d2h_bytes_per_step": 2 * fbytes}

    extras = {}
    if not a.no_extras and rank == 0:
        del hu, hp, hc, ou, op
        extras = _extras(torch, W, B, Level, arith, stream,
                         which=[x for x in a.extras.split(",") if x])

    cpu = None
    if rank == 0 and ws == 1 and not a.no_cpu:
        # a bounded sample of about 12 s of oracle work: the step count is
        # calibrated by a 2-step run (counted in the sample)
        r0, used, dt0 = _oracle_rate(inst, 2)
        nmore = max(1, int(round((CPU_SAMPLE_S - dt0) * r0 / npts)))
        r1, used, dt1 = _oracle_rate(inst, nmore)
        nall = 2 + nmore
        r = npts * nall / (dt0 + dt1)
        cpu = {"value": r, "unit": UNIT, "cores": used, "kind": "oracle",
               "sample": "%d RK4 steps of the same 256^3 workload (%.1f s)" % (nall, dt0 + dt1)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * t / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_LABEL[a.arith],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "points": npts, "rk4_steps_per_step": nsub,
                       "arith": a.arith, "mode": "batched persistent launch, CUDA graph per "
                                                  "RK4 step",
                       "stages_per_pass": form,
                       "pass_kernel": ("warp-specialised" if lev.get_pass_kernel() ==
                                       B.SC_PASS_WARP_SPECIALISED else "one-role")
                       if form == 2 else None,
                       "tiles": [list(lev.get_tuning(c)) for c in range(lev.size_classes()[0])],
                       "l2": "inputs larger than L2 (fields 7 x %d MB)" % (fbytes >> 20),
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "kernel": kname,
                         "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm if hbm else None, "traffic": traffic,
                         "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
                         "bytes_per_launch": bytes_launch,
                         "launches": nlaunch, "avg_launch_ms": avg_ms,
                         "gather_avg_launch_ms": gather_ms / max(gather_n, 1),
                         "fp64_tflops_est": fp64_achieved,
                         "fp64_fraction_of_measured": fp64_achieved / (2e-3 * FP64_FMA_RATE_G),
                         "classic_equivalent_gbs": value * BYTES_PER_POINT_STEP_CLASSIC / 1e9,
                         "hbm_fraction_of_nominal_7900": achieved / 7900.0,
                         "kernel_hash": khash,
                         "note": ("two RK4 stages per pass halve the DRAM bytes of a step; "
                                  "in the warp-specialised kernels producer warps form the "
                                  "fixed-point sums while consumer warps run the FP64 "
                                  "epilogue, so the integer and FP64 pipes work at the same "
                                  "time; what remains is memory latency and issue; "
                                  "classic_equivalent_gbs is the rate times the 304 B per "
                                  "point and step of an unfused stage form")
                         if form == 2 else "one stage per pass, HBM-bound"},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "step_ms": ({"best": per_step[0], "median": per_step[len(per_step) // 2],
                         "steps": len(per_step)} if per_step else None),
            "clocks": clk,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    a = _args()
    ws, rank, local = _dist()
    if a.impl == "reference":
        run_reference(a, ws, rank)
        return
    run_ours(a, ws, rank, local)


if __name__ == "__main__":
    main()
