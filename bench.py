#!/usr/bin/env python
"""Benchmark of the split-preconditioned fixed-point solver on one GB300.

Workload: the 3-D Helmholtz medium of size 256^3 (refractive index 1-1.5
from a seeded smoothed random field, sigma 6 px, plus spheres of n = 1.45,
absorbing layer 32 px per face, Gaussian beam source), pixel = lambda/4,
complex64, solved to a relative preconditioned residual of 1e-6.

One step = create the solver (validation, alpha, scratch) + solve to 1e-6
(reference norm, iterations, refinement) + destroy, inputs resident in
HBM.  `value` = iterations per second over the timed steps (all ranks);
`ms_per_step` = seconds to residual 1e-6 per solve.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores instead (the
reference arm: there is no reference implementation, only the paper).
Multi-GPU runs are independent replicas (the solve does not shard).
"""

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "256³ Helmholtz: s to residual 1e-6, iter/s, % HBM roofline; plain vs chosen"
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=256)
    p.add_argument("--ndim", type=int, default=3, choices=[2, 3],
                   help="2: the 2-D n x n Helmholtz medium (sigma 4 px, ABL n/8) instead of the 3-D one")
    p.add_argument("--workload", default="helmholtz", choices=["helmholtz", "diffusion"])
    p.add_argument("--nz", type=int, default=0,
                   help="3-D slab nz x n x n instead of n^3 (small profiling cases)")
    p.add_argument("--tol", type=float, default=1e-6)
    p.add_argument("--maxit", type=int, default=20000)
    p.add_argument("--schedule", type=int, default=0)
    p.add_argument("--plain", action="store_true", help="time the plain FP32 iteration")
    p.add_argument("--cols-tile", type=int, default=0,
                   help="columns per staged strided-axis tile (16, 32; 0 = library default)")
    p.add_argument("--tc-dft", action="store_true",
                   help="256-point strided-axis transforms on the tensor cores")
    p.add_argument("--no-tma", action="store_true",
                   help="strided-axis passes without TMA staging (comparison)")
    p.add_argument("--cpu-iters", type=int, default=10)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip e2e, plain and roofline legs")
    p.add_argument("--batch", type=int, default=64,
                   help="problems of the batched leg (2-D 128x128 media; 0 skips it)")
    p.add_argument("--batch-n", type=int, default=128)
    p.add_argument("--mixed", type=int, default=512,
                   help="problems of the mixed-size 2-D batch leg (0 skips it)")
    p.add_argument("--fno-train", type=int, default=4096,
                   help="solved 128x128 media the warm-start network trains on (0 skips)")
    p.add_argument("--fno-epochs", type=int, default=20)
    p.add_argument("--fno-test", type=int, default=256, help="held-out media")
    p.add_argument("--no-variants", action="store_true", help="skip the block-variant leg")
    p.add_argument("--no-diffusion", action="store_true",
                   help="skip the 3-D diffusion leg of the Helmholtz line")
    return p.parse_args()


def reduce_timing(elapsed_ms, units, dist, device):
    """Whole-job timing over the ranks: the slowest rank's time and the sum
    of the units every rank processed (identity without a process group)."""
    if dist is None:
        return float(elapsed_ms), int(units)
    import torch
    t = torch.tensor([float(elapsed_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(units)], device=device, dtype=torch.float64)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(c.item()))


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(args, seed=0):
    from paper_2207_14222_gb300 import inputs
    if args.ndim == 2:
        if args.workload == "helmholtz":
            return inputs.helmholtz_2d(args.n, seed=seed, abl_width=max(4, args.n // 8))
        return inputs.random_diffusion((args.n, args.n), seed, sigma_px=4.0)
    if args.nz:
        # profiling slabs: nz x n x n, the same medium statistics
        shape = (args.nz, args.n, args.n)
        if args.workload == "helmholtz":
            return inputs.random_helmholtz(shape, seed, sigma_px=6.0 * args.n / 256,
                                           amplitude=0.3, abl_width=max(2, args.nz // 8))
        return inputs.random_diffusion(shape, seed, sigma_px=6.0 * args.n / 256,
                                       median_eta=0.01)
    if args.workload == "helmholtz":
        return inputs.helmholtz_3d(args.n, seed=seed)
    return inputs.diffusion_3d(args.n, seed=seed)


def workload_name(args):
    if args.nz:
        return "%s3d_%dx%dx%d" % (args.workload, args.nz, args.n, args.n)
    return "%s%dd_%d" % (args.workload, args.ndim, args.n)


# ---------------------------------------------------------------- clocks ---

class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.gpu_id is not None:
                cmd += ["-i", str(self.gpu_id)]
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons, n = [], [], set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            n += 1
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": n}


def gpu_smi_id(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# ------------------------------------------------------------- roofline ---

def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# FP32 lanes per SM (Blackwell): the ALU peak of the on-chip schedule, whose
# fields stay in shared memory between iterations (no HBM traffic to bound it).
FP32_LANES_PER_SM = 128
NOMINAL_SM_MHZ = 2070.0


def onchip_flop_per_point(n):
    """Algorithmic flops per grid point of one on-chip iteration on an n x n
    grid: forward and inverse 2-D FFT at 5 log2(N) each (N = n^2), plus 40
    pointwise ((1 - V) x + y: 8; multiplier 1/(N (Lhat + 1)): 14 with the
    complex product; Delta = (1 - V)(u - x): 8; update 4; |Delta|^2: 4;
    rounded up)."""
    return 2 * 5 * math.log2(n * n) + 40


def onchip_roofline(passes, problems, n, torch, dev, sm_mhz=None):
    """ALU roofline of an on-chip iteration (one kernel per phase; its mean
    per iteration from usp_time_passes)."""
    ms = sum(p["ms"] for p in passes)
    flop = onchip_flop_per_point(n) * n * n * problems
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = sm_mhz or NOMINAL_SM_MHZ
    peak = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    achieved = flop / (ms * 1e-3) / 1e12
    return {"bound": "alu", "kernel": "onchip_iteration", "iteration_ms": ms,
            "flop_per_iteration": flop, "achieved_tflops": achieved,
            "peak_tflops": peak, "peak_source": "%d SMs x %d FP32 lanes x 2 x %.0f MHz"
            % (sms, FP32_LANES_PER_SM, mhz), "frac": achieved / peak}


def schedule_efficiency(passes, points, vreal, iteration_ms, peak):
    """The iteration's floor -- read x, y and V, write x: 32 bytes per point
    (28 with a real V) -- against the bytes the schedule moves per iteration:
    their ratio, and the iterations/s the floor would allow at the peak."""
    floor = 28.0 if vreal else 32.0
    sched = sum(p["bytes"] for p in passes) / points
    return {"floor_bytes_per_point": floor, "schedule_bytes_per_point": sched,
            "schedule_efficiency": floor / sched if sched > 0 else None,
            "floor_iter_per_s": peak * 1e9 / (floor * points),
            "iter_per_s_at_iteration_ms": 1e3 / iteration_ms}


# Sources of the 3-D pass kernels (pencil and split-y schedules) whose ncu
# traffic is recorded.
PENCIL_SOURCES = ("fft_core.cuh", "iteration_state.cuh", "kernels.h", "pencil_core.cuh", "pencil_kernels.cu",
                  "tma.cuh", "tma_kernels.cu", "split3d_kernels.cu")


def kernel_sources_sha():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2207_14222_gb300", "csrc")
    for f in PENCIL_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel):
    """DRAM bytes per launch recorded from an ncu capture in profiles/, valid
    only if the kernel sources are unchanged since (line format:
    `bench-traffic: <pass> <bytes per launch> <sources sha>`)."""
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return None
    sha = kernel_sources_sha()
    for f in sorted(os.listdir(d)):
        if not f.endswith((".md", ".txt")):
            continue
        for line in open(os.path.join(d, f)):
            m = re.match(r"\s*bench-traffic:\s*(\S+)\s+([0-9.eE+]+)\s+(\S+)", line)
            if m and m.group(1) == kernel and m.group(3) == sha:
                return float(m.group(2))
    return None


# ------------------------------------------------------------ our arm ---

def run_ours(args):
    import torch
    from paper_2207_14222_gb300 import canon
    from paper_2207_14222_gb300.solver import Solver, kernel_launches

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    prob = workload(args)
    cf = canon.canonical(prob)
    shape = cf["V"].shape
    V = torch.from_numpy(cf["V"]).to(dev)
    y = torch.from_numpy(cf["y"]).to(dev)
    x = torch.empty_like(y)

    def step():
        with Solver(shape, cf["a"], cf["b"], V, plain=args.plain, schedule=args.schedule,
                    no_tma=args.no_tma, cols_tile=args.cols_tile, tc_dft=args.tc_dft) as s:
            _, r = s.solve(y, x=x, tol=args.tol, maxit=args.maxit)
        return r

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_smi_id(torch, dev))
    sampler.start()
    l0 = kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    res = [step() for _ in range(args.steps)]
    e1.record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches = kernel_launches() - l0
    clocks = sampler.stop()
    elapsed_ms = e0.elapsed_time(e1)
    iters = sum(r["iterations"] for r in res)
    elapsed_ms, iters_all = reduce_timing(elapsed_ms, iters, dist, dev)
    value = iters_all / (elapsed_ms / 1e3)
    ms_per_step = elapsed_ms / args.steps

    extras = {}
    if not args.no_extras:
        extras = extras_legs(args, torch, dev, cf, V, y, shape, Solver, res[-1]["iterations"])
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, prob)

    if rank == 0:
        last = res[-1]
        line = {
            "metric": METRIC,
            "value": value,
            "unit": "iter/s",
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_per_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "config": {
                "workload": workload_name(args),
                "grid": list(shape),
                "tol": args.tol,
                "mode": "plain" if args.plain else "fp32+refinement (residual in double-float)",
                "schedule": ["auto", "pencil", "fused", "on-chip", "split"][args.schedule],
                "tma": not args.no_tma,
                "cols_tile": args.cols_tile or "default",
                "tc_dft": args.tc_dft,
                "step": "create + solve to tol + destroy",
                "l2": ("inputs 384 MiB > L2, no flush" if args.ndim == 3 else
                       "fields resident on chip between iterations"),
                "replicas": ws,
            },
            "s_to_residual": ms_per_step / 1e3,
            "iterations": last["iterations"],
            "refinements": last["refinements"],
            "final_rel_residual": last["final_rel_residual"],
            "converged": bool(last["converged"]),
            "gpu_launches": launches,
            "clocks": clocks,
        }
        line.update(extras)
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def extras_legs(args, torch, dev, cf, V, y, shape, Solver, ref_iters):
    out = {}
    # per-kernel durations (CUDA events on the solver's stream) -> roofline
    xt = torch.empty_like(y)
    with Solver(shape, cf["a"], cf["b"], V, schedule=args.schedule, no_tma=args.no_tma,
                cols_tile=args.cols_tile, tc_dft=args.tc_dft) as s:
        s.solve(y, x=xt, tol=0.0, maxit=5)  # warm
        passes = s.time_passes(y, xt, iters=20)
    per_it_ms = sum(p["ms"] for p in passes)
    dom = max(passes, key=lambda p: p["ms"])
    peak, kind = measured_hbm_peak()
    achieved = dom["bytes"] / (dom["ms"] * 1e-3) / 1e9
    if dom["name"] == "onchip_iteration":
        out["roofline"] = onchip_roofline(passes, 1, shape[0], torch, dev)
    else:
        out["roofline"] = {
            "bound": "hbm", "kernel": dom["name"], "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "peak_source": kind,
            "traffic": recorded_traffic(dom["name"]),
            "bytes_per_launch": dom["bytes"], "ms_per_launch": dom["ms"],
            "iteration_ms": per_it_ms,
            "iteration_frac": sum(p["bytes"] for p in passes) / (per_it_ms * 1e-3) / 1e9 / peak,
            "passes": [{"name": p["name"], "ms": round(p["ms"], 5),
                        "GBps": round(p["bytes"] / (p["ms"] * 1e-3) / 1e9, 1)} for p in passes],
        }
        out["roofline"].update(schedule_efficiency(passes, int(np.prod(shape)), V.dtype == torch.float32,
                                                   per_it_ms, peak))
        if dom["name"] == "split_rows_full":
            out["roofline"]["bytes_note"] = (
                "split_rows_full reads only the source rows that hold nonzero values: 40 B/pt "
                "(36 with a real V) plus 8 B/pt per nonzero source row; 48 B/pt with a dense source")
    # end to end through the host API: pinned V, y in; x out
    Vh = V.cpu().pin_memory()
    yh = y.cpu().pin_memory()
    xh = torch.empty_like(yh).pin_memory()
    t_it, t_s = 0, 0.0
    steps = max(1, min(args.steps, 3))
    for k in range(steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Vd = Vh.to(dev, non_blocking=True)
        with Solver(shape, cf["a"], cf["b"], Vd, plain=args.plain, schedule=args.schedule) as s:
            _, r = s.solve_host(yh, xh, tol=args.tol, maxit=args.maxit)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        del Vd
        if k > 0:  # first one is warm-up
            t_it += r["iterations"]
            t_s += dt
    out["e2e"] = {"value": t_it / t_s, "unit": "iter/s",
                  "h2d_bytes_per_step": int(Vh.numel() * Vh.element_size() + yh.numel() * 8),
                  "d2h_bytes_per_step": int(xh.numel() * 8),
                  "s_per_solve": t_s / steps}
    # plain Algorithm 1 (no refinement) on the same problem: its FP32 floor
    if not args.plain:
        xp = torch.empty_like(y)
        with Solver(shape, cf["a"], cf["b"], V, plain=True, schedule=args.schedule) as s:
            maxit = 4 * max(ref_iters, 250)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, r = s.solve(y, x=xp, tol=args.tol, maxit=maxit)
            dt = time.perf_counter() - t0
            h = s.history()
        out["plain"] = {"reached_tol": bool(r["converged"]), "iterations": r["iterations"],
                        "min_rel_residual": float(h.min()), "argmin": int(h.argmin()) + 1,
                        "iter_per_s": r["iterations"] / dt,
                        "s_to_min_residual": dt * (int(h.argmin()) + 1) / r["iterations"]}
    out["library_comparator"] = cufft_leg(torch, dev, cf, V, y, shape)
    if args.ndim == 3 and args.workload == "helmholtz" and not args.no_diffusion:
        out["diffusion3d_%d" % args.n] = diffusion3d_leg(args, torch, dev)
    out["helmholtz2d_128"] = helmholtz2d_leg(args, torch, dev)
    if args.batch > 0:
        out["batched"] = batched_leg(args, torch, dev)
    if args.mixed > 0:
        out["mixed_batch"] = mixed_batch_leg(args, torch, dev)
    if args.fno_train > 0:
        out["fno_warm_start"] = fno_leg(args, torch, dev)
    if not args.no_variants:
        out["variants"] = variants_leg(args, torch, dev)
    return out


def diffusion3d_leg(args, torch, dev):
    """The second 3-D workload: steady diffusion on an n^3 grid (log-normal
    absorption, median 0.01 per px, sigma_log 0.5, smoothed over 6 px; D = 1;
    centre point source; real V), solved to the bench tolerance the same way
    as the main line (create + solve + destroy per step, CUDA events, inputs
    resident: 320 MiB > L2, no flush).  Also: plain FP32 Algorithm 1, and the
    per-pass roofline on the real-V floor (28 B per point) and on the
    schedule's bytes."""
    from paper_2207_14222_gb300 import canon, inputs
    from paper_2207_14222_gb300.solver import Solver
    n = args.n
    cf = canon.canonical(inputs.diffusion_3d(n, seed=0))
    shape = cf["V"].shape
    V = torch.from_numpy(cf["V"]).to(dev)
    y = torch.from_numpy(cf["y"]).to(dev)
    x = torch.empty_like(y)

    def step(plain=False):
        with Solver(shape, cf["a"], cf["b"], V, dx=cf["dx"], plain=plain,
                    schedule=args.schedule) as s:
            _, r = s.solve(y, x=x, tol=args.tol, maxit=args.maxit)
        return r

    out = {"workload": "diffusion3d_%d" % n, "grid": list(shape), "tol": args.tol,
           "V": "float32 (real)", "step": "create + solve to tol + destroy",
           "l2": "inputs 320 MiB > L2, no flush"}
    for name, plain in (("chosen", False), ("plain", True)):
        for _ in range(3):
            step(plain)
        torch.cuda.synchronize()
        reps = max(args.steps, 5)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rs = [step(plain) for _ in range(reps)]
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        r = rs[-1]
        out[name] = {"s_to_residual": ms / 1e3, "iterations": r["iterations"],
                     "refinements": r["refinements"], "converged": bool(r["converged"]),
                     "final_rel_residual": r["final_rel_residual"],
                     "iter_per_s": sum(q["iterations"] for q in rs) / (reps * ms / 1e3)}
    with Solver(shape, cf["a"], cf["b"], V, dx=cf["dx"], schedule=args.schedule) as s:
        s.solve(y, x=x, tol=0.0, maxit=5)
        passes = s.time_passes(y, x, iters=20)
    per_it_ms = sum(p["ms"] for p in passes)
    peak, kind = measured_hbm_peak()
    dom = max(passes, key=lambda p: p["ms"])
    achieved = dom["bytes"] / (dom["ms"] * 1e-3) / 1e9
    out["roofline"] = {
        "bound": "hbm", "kernel": dom["name"], "achieved": achieved, "peak": peak,
        "unit": "GB/s", "frac": achieved / peak, "peak_source": kind,
        "iteration_ms": per_it_ms,
        "iteration_frac": sum(p["bytes"] for p in passes) / (per_it_ms * 1e-3) / 1e9 / peak,
        "passes": [{"name": p["name"], "ms": round(p["ms"], 5),
                    "GBps": round(p["bytes"] / (p["ms"] * 1e-3) / 1e9, 1)} for p in passes]}
    out["roofline"].update(schedule_efficiency(passes, int(np.prod(shape)), True, per_it_ms, peak))
    out["roofline"]["floor_frac"] = (out["roofline"]["floor_bytes_per_point"] * np.prod(shape)
                                     / (per_it_ms * 1e-3) / 1e9 / peak)
    return out


def variants_leg(args, torch, dev):
    """The block forms: the antisymmetrised Helmholtz problem with gain on
    128 x 128 (K = 2; on chip, and with the passes for comparison) and
    flux-form diffusion with variable D on 128^3 (K = 4), plain FP32
    Algorithm 1 to 1e-5.  Algorithmic bytes per point and iteration of the
    passes: pre (read K x, K y, V; write K t) + each transform pass (read and
    write K planes) + multiply (K read, K write) + post (read K u, K x, V;
    write K x)."""
    from paper_2207_14222_gb300 import canon, inputs
    from paper_2207_14222_gb300.solver import VariantSolver
    peak, _ = measured_hbm_peak()
    out = {}
    cases = []
    # the antisymmetrised form contracts slowly (its rate follows the
    # singular values of A0, not its numerical range): a 128^2 medium with
    # n - 1 in [0, 0.1] and |kappa| <= 0.05
    g = inputs.gain_helmholtz((128, 128), 0, contrast=0.1, gain=0.05, sigma_px=4.0)
    cases.append(("antisymmetric_helmholtz_128x128", (128, 128),
                  canon.antisymmetric(g["k2"], g["S"]), 2, 8))
    d = inputs.variable_diffusion((128, 128, 128), 0, sigma_px=4.0)
    cases.append(("flux_diffusion_128^3", (128, 128, 128),
                  canon.flux_diffusion(d["eta"], d["D"], np.real(d["S"])), 4, 8))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    for name, shape, cp, K, vb in cases:
        N = int(np.prod(shape))
        passes = 2 * len(shape)
        bpp = (24 * K + vb) + passes * 16 * K + 16 * K + (24 * K + vb)
        V = torch.from_numpy(cp["V"]).to(dev)
        y = torch.from_numpy(cp["y"]).to(dev)
        maxit = max(args.maxit, 100000)
        # square 2-D grids up to 128^2 run on chip by default; the passes beside them
        scheds = [("onchip", 0), ("passes", 1)] if len(shape) == 2 and shape[0] == shape[1] else [("passes", 0)]
        res = {}
        for label, sched in scheds:
            with VariantSolver(shape, cp["kind"], cp["params"], V, schedule=sched) as s:
                s.solve(y, tol=1e-5, maxit=50)       # warm-up
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, r = s.solve(y, tol=1e-5, maxit=maxit)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
            d = {"iterations": r["iterations"], "converged": bool(r["converged"]), "s_to_1e-5": dt,
                 "iter_per_s": r["iterations"] / dt}
            if label == "onchip":
                # ALU bound: K forward + inverse 2-D FFTs and the block pointwise steps
                flop = (K * 2 * 5 * math.log2(N) + 40 * K) * N
                ach = flop * r["iterations"] / dt / 1e12
                peak_t = sms * FP32_LANES_PER_SM * 2 * NOMINAL_SM_MHZ * 1e6 / 1e12
                d.update({"bound": "alu", "flop_per_iteration": flop, "achieved_tflops": ach,
                          "peak_tflops": peak_t, "frac": ach / peak_t})
            else:
                gbs = bpp * N * r["iterations"] / dt / 1e9
                d.update({"bound": "hbm", "bytes_per_point_iter": bpp, "GBps": gbs, "frac_of_peak": gbs / peak})
            res[label] = d
        entry = {"K": K}
        entry.update(res[scheds[0][0]])
        if len(scheds) > 1:
            entry["passes"] = res["passes"]
            entry["speedup_vs_passes"] = res["passes"]["s_to_1e-5"] / res["onchip"]["s_to_1e-5"]
        out[name] = entry
    return out


def fno_leg(args, torch, dev):
    """The learned warm start on the 2-D 128x128 medium distribution: train
    the network (width 32, 4 layers, 16 x 16 modes) on media solved by the
    batch solver, then solve held-out media to the tolerance from zero and
    from the network's estimate (inference included in the time)."""
    from paper_2207_14222_gb300 import canon, inputs
    from paper_2207_14222_gb300.fno import FNO, features
    from paper_2207_14222_gb300.solver import BatchSolver
    n, bs = 128, 32

    def dataset(seeds):
        probs = [inputs.helmholtz_2d(n, seed=s) for s in seeds]
        cfs = [canon.canonical(p) for p in probs]
        V = torch.from_numpy(np.stack([cf["V"] for cf in cfs])).to(dev)
        y = torch.from_numpy(np.stack([cf["y"] for cf in cfs])).to(dev)
        a = torch.from_numpy(np.stack([features(p) for p in probs])).to(dev)
        return cfs, V, y, a

    def solve(cfs, V, y, x0=None):
        with BatchSolver((n, n), [cf["a"] for cf in cfs], [cf["b"] for cf in cfs], V) as s:
            x, res = s.solve(y, x=x0, use_x0=x0 is not None, tol=args.tol, maxit=args.maxit)
        return x, res

    t0 = time.perf_counter()
    cfs, V, y, a = dataset(range(10000, 10000 + args.fno_train))
    xs, _ = solve(cfs, V, y)
    del V, y
    t_data = time.perf_counter() - t0
    losses = []
    with FNO(n, n, width=32, layers=4, modes=16, max_batch=bs, seed=0) as net:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for ep in range(args.fno_epochs):
            perm = torch.randperm(args.fno_train, generator=torch.Generator().manual_seed(ep)).to(dev)
            ls = [net.train_step(a[perm[k:k + bs]], xs[perm[k:k + bs]],
                                 lr=2e-3 * 0.5 ** (ep * 3 // max(args.fno_epochs, 1)))
                  for k in range(0, args.fno_train - bs + 1, bs)]
            losses.append(float(np.mean(ls)))
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        tcfs, tV, ty, ta = dataset(range(90000, 90000 + args.fno_test))
        solve(tcfs, tV, ty)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xz, rz = solve(tcfs, tV, ty)
        torch.cuda.synchronize()
        t_zero = time.perf_counter() - t0
        t0 = time.perf_counter()
        x0 = torch.cat([net.predict(ta[k:k + bs]) for k in range(0, args.fno_test, bs)])
        torch.cuda.synchronize()
        t_inf = time.perf_counter() - t0
        xw, rw = solve(tcfs, tV, ty, x0.clone())
        torch.cuda.synchronize()
        t_warm = time.perf_counter() - t0
    err = torch.linalg.vector_norm(x0 - xz, dim=(1, 2)) / torch.linalg.vector_norm(xz, dim=(1, 2))
    iz = np.array([r["iterations"] for r in rz])
    iw = np.array([r["iterations"] for r in rw])
    return {"train_media": args.fno_train, "epochs": args.fno_epochs, "test_media": args.fno_test,
            "data_s": t_data, "train_s": t_train, "loss_first_last": [losses[0], losses[-1]],
            "median_rel_error_x0": float(err.median()),
            "iterations_zero_median": float(np.median(iz)),
            "iterations_warm_median": float(np.median(iw)),
            "iterations_saved_total_frac": float(1 - iw.sum() / iz.sum()),
            "converged_warm": int(sum(r["converged"] for r in rw)),
            "s_zero": t_zero, "s_warm_incl_inference": t_warm, "s_inference": t_inf,
            "speedup": t_zero / t_warm}


def mixed_batch_leg(args, torch, dev):
    """The mixed-size workload: 2-D problems of sides 64-512 (radix 2 and
    3), Helmholtz and diffusion alternating, each with its own medium; one
    batch solver per side, autotuned, all sides solved concurrently
    (usp_solve_many) vs one solver per problem in turn."""
    from paper_2207_14222_gb300 import canon, inputs
    from paper_2207_14222_gb300.solver import BatchSolver, Solver, solve_many
    groups = {}
    for i in range(args.mixed):
        prob = inputs.batch_problem(i)
        cf = canon.canonical(prob)
        groups.setdefault(prob["S"].shape[0], []).append(cf)
    sides = sorted(groups)
    Vg = {n: torch.from_numpy(np.stack([cf["V"].astype(np.complex64) for cf in groups[n]])).to(dev)
          for n in sides}
    yg = {n: torch.from_numpy(np.stack([cf["y"] for cf in groups[n]])).to(dev) for n in sides}

    def together(which=None):
        which = sides if which is None else which
        solvers = [BatchSolver((n, n), [cf["a"] for cf in groups[n]],
                               [cf["b"] for cf in groups[n]], Vg[n]) for n in which]
        try:
            for sv, n in zip(solvers, which):
                sv.autotune(yg[n], iters=3)
            _, res = solve_many(solvers, [yg[n] for n in which], tol=args.tol,
                                maxit=args.maxit)
        finally:
            for sv in solvers:
                sv.close()
        return [r for lst in res for r in lst]

    def one_by_one():
        res = []
        for n in sides:
            for j, cf in enumerate(groups[n]):
                with Solver((n, n), cf["a"], cf["b"], Vg[n][j]) as sv:
                    _, r = sv.solve(yg[n][j], tol=args.tol, maxit=args.maxit)
                res.append(r)
        return res

    pts = {n: n * n for n in sides}
    # per side: one batched iteration's passes (CUDA events) -> roofline
    peak, _ = measured_hbm_peak()
    per_side = {}
    for n in sides:
        with BatchSolver((n, n), [cf["a"] for cf in groups[n]], [cf["b"] for cf in groups[n]],
                         Vg[n]) as sv:
            xt = torch.empty_like(yg[n])
            sv.solve(yg[n], x=xt, tol=0.0, maxit=3)
            ps = sv.time_passes(yg[n], xt, iters=10)
        ms = sum(p["ms"] for p in ps)
        if ps[0]["name"] == "onchip_iteration":
            rf = onchip_roofline(ps, len(groups[n]), n, torch, dev)
            per_side[str(n)] = {"iteration_ms": round(ms, 5), "schedule": "on-chip",
                                "bound": "alu", "frac": round(rf["frac"], 3)}
        else:
            per_side[str(n)] = {"iteration_ms": round(ms, 5), "schedule": "pencil", "bound": "hbm",
                                "frac": round(sum(p["bytes"] for p in ps) / (ms * 1e-3) / 1e9 / peak, 3)}
    out = {"problems": args.mixed, "tol": args.tol, "per_side_iteration": per_side,
           "sides": {str(n): len(groups[n]) for n in sides},
           "points": int(sum(pts[n] * len(groups[n]) for n in sides)),
           "step": "create + autotune + solve every problem to tol + destroy"}
    for name, fn in (("concurrent_batches", together), ("one_by_one", one_by_one)):
        fn()  # warm-up (also fills the autotuner's cache)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = fn()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        its = [r["iterations"] for r in res]
        out[name] = {"s": dt, "problem_iter_per_s": sum(its) / dt,
                     "converged": sum(int(r["converged"]) for r in res),
                     "iterations_min_max": [min(its), max(its)]}
    out["speedup"] = out["one_by_one"]["s"] / out["concurrent_batches"]["s"]
    # the critical path: each side's batch alone, and the on-chip sides
    # (one launch per phase each) against the sides on the passes
    def timed(which):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        together(which)
        torch.cuda.synchronize()
        return time.perf_counter() - t0
    out["side_alone_s"] = {str(n): round(timed([n]), 5) for n in sides}
    small = [n for n in sides if per_side[str(n)]["schedule"] == "on-chip"]
    large = [n for n in sides if n not in small]
    if small and large:
        out["onchip_sides_together_s"] = round(timed(small), 5)
        out["pass_sides_together_s"] = round(timed(large), 5)
    return out


def cufft_leg(torch, dev, cf, V, y, shape, iters=20):
    """The same FP32 iteration written with torch.fft (cuFFT) and torch
    elementwise ops on the same GPU: the library comparator (not the
    product path, which runs only the library's own kernels)."""
    ks = [torch.fft.fftfreq(n, d=cf["dx"], device=dev, dtype=torch.float64) * 2 * np.pi
          for n in shape]
    p2 = sum(torch.meshgrid(*[k * k for k in ks], indexing="ij"))
    a, b = complex(cf["a"]), complex(cf["b"])
    mult = (1.0 / (a * p2 + b + 1.0)).to(torch.complex64)
    del p2
    Bm = (1 - V.to(torch.complex64))
    alpha = float(np.min(np.real(1.0 / Bm.cpu().numpy())))
    x = torch.zeros_like(y)

    def it():
        t = Bm * x + y
        u = torch.fft.ifftn(torch.fft.fftn(t) * mult)
        d = Bm * (u - x)
        x.add_(d, alpha=alpha)
        return torch.linalg.vector_norm(d)

    for _ in range(3):
        it()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(iters):
        it()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / iters
    return {"what": "torch.fft (cuFFT) + torch elementwise ops, complex64, same iteration",
            "iter_per_s": 1e3 / ms, "ms_per_iter": ms}


def helmholtz2d_leg(args, torch, dev):
    """One 2-D 128 x 128 Helmholtz problem (sigma 4 px, amplitude 0.3, ABL 16
    px, centre point source) to the bench tolerance with refinement: the
    on-chip schedule (automatic for this grid) against the pencil passes."""
    from paper_2207_14222_gb300 import canon, inputs
    from paper_2207_14222_gb300.solver import Solver
    n = 128
    cf = canon.canonical(inputs.helmholtz_2d(n, seed=0))
    V = torch.from_numpy(np.asarray(cf["V"], np.complex64)).to(dev)
    y = torch.from_numpy(np.asarray(cf["y"], np.complex64)).to(dev)
    out = {"grid": [n, n], "tol": args.tol, "step": "solve to tol (solver created once)"}
    for name, sched in (("onchip", 3), ("pencil", 1)):
        with Solver((n, n), cf["a"], cf["b"], V, dx=cf["dx"], schedule=sched) as s:
            x = torch.empty_like(y)
            for _ in range(3):
                s.solve(y, x=x, tol=args.tol, maxit=args.maxit)
            torch.cuda.synchronize()
            reps = 20
            t0 = time.perf_counter()
            for _ in range(reps):
                _, r = s.solve(y, x=x, tol=args.tol, maxit=args.maxit)
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t0) / reps
            ps = s.time_passes(y, x, iters=200)
        d = {"s_to_residual": dt, "iterations": r["iterations"], "refinements": r["refinements"],
             "converged": bool(r["converged"]), "us_per_iteration": 1e3 * sum(p["ms"] for p in ps)}
        if sched == 3:
            d["roofline"] = onchip_roofline(ps, 1, n, torch, dev)
        out[name] = d
    out["speedup"] = out["pencil"]["s_to_residual"] / out["onchip"]["s_to_residual"]
    return out


def batched_leg(args, torch, dev):
    """Many small 2-D problems (the 128x128 medium distribution, one seed
    each): solved together by one batch solver vs one solver per problem,
    both to the same tolerance with refinement."""
    from paper_2207_14222_gb300 import canon, inputs
    from paper_2207_14222_gb300.solver import BatchSolver, Solver
    n, B = args.batch_n, args.batch
    cfs = [canon.canonical(inputs.helmholtz_2d(n, seed=1000 + j, abl_width=max(4, n // 8)))
           for j in range(B)]
    V = torch.from_numpy(np.stack([cf["V"] for cf in cfs])).to(dev)
    y = torch.from_numpy(np.stack([cf["y"] for cf in cfs])).to(dev)
    a = [cf["a"] for cf in cfs]
    b = [cf["b"] for cf in cfs]

    def batched():
        with BatchSolver((n, n), a, b, V) as s:
            _, res = s.solve(y, tol=args.tol, maxit=args.maxit)
        return res

    def one_by_one():
        res = []
        for j in range(B):
            with Solver((n, n), a[j], b[j], V[j]) as s:
                _, r = s.solve(y[j], tol=args.tol, maxit=args.maxit)
            res.append(r)
        return res

    out = {"problems": B, "grid": [n, n], "tol": args.tol,
           "step": "create + solve every problem to tol + destroy"}
    # per-pass durations of one batched iteration (CUDA events) -> roofline
    with BatchSolver((n, n), a, b, V) as s:
        xt = torch.empty_like(y)
        s.solve(y, x=xt, tol=0.0, maxit=3)
        passes = s.time_passes(y, xt, iters=20)
    peak, _ = measured_hbm_peak()
    it_ms = sum(p["ms"] for p in passes)
    if passes[0]["name"] == "onchip_iteration":
        out["roofline"] = onchip_roofline(passes, B, n, torch, dev)
    else:
        out["roofline"] = {"iteration_ms": it_ms,
                           "iteration_frac": sum(p["bytes"] for p in passes) / (it_ms * 1e-3) / 1e9 / peak,
                           "passes": [{"name": p["name"], "ms": round(p["ms"], 5),
                                       "GBps": round(p["bytes"] / (p["ms"] * 1e-3) / 1e9, 1)}
                                      for p in passes]}
    for name, fn in (("batched", batched), ("one_by_one", one_by_one)):
        fn()  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = fn()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        its = [r["iterations"] for r in res]
        out[name] = {"s": dt, "problem_iter_per_s": sum(its) / dt,
                     "converged": sum(int(r["converged"]) for r in res),
                     "iterations_min_max": [min(its), max(its)]}
    out["speedup"] = out["one_by_one"]["s"] / out["batched"]["s"]
    return out


# ------------------------------------------------------ CPU (oracle) arm ---

def _oracle_setup(prob):
    from oracle import canon as ocanon
    from oracle import usp_oracle as uo
    cf = ocanon.canonical(prob)
    Lh = uo.lhat(cf["V"].shape, cf["dx"], cf["a"], cf["b"])
    return cf, Lh, uo


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _time_oracle(uo, cf, Lh, alpha, iters, workers, warm=1):
    """Seconds per iteration of the FP64 oracle's Algorithm 1 (its FFT on
    ``workers`` host threads), after ``warm`` untimed iterations."""
    import scipy.fft as sfft
    with sfft.set_workers(workers):
        x, _ = uo.iterate(cf["V"], cf["y"], Lh, alpha, warm, ref_norm=1.0)
        t0 = time.perf_counter()
        uo.iterate(cf["V"], cf["y"], Lh, alpha, iters, x0=x, ref_norm=1.0)
        return (time.perf_counter() - t0) / iters


def cpu_baseline(args, prob, iters=None):
    """The FP64 oracle as it stands, a bounded sample of the same workload:
    all host cores (its FFT threaded by scipy.fft), and one core beside it."""
    iters = iters or args.cpu_iters
    cf, Lh, uo = _oracle_setup(prob)
    alpha = uo.alpha_star(cf["V"])
    cores = _host_cores()
    dt = _time_oracle(uo, cf, Lh, alpha, iters, cores)
    dt1 = _time_oracle(uo, cf, Lh, alpha, max(2, iters // 5), 1, warm=0)
    return {"value": 1.0 / dt, "unit": "iter/s", "cores": cores, "kind": "oracle",
            "sample": "%d timed iterations (after one untimed) of Algorithm 1 on the %s "
                      "workload, FP64 oracle with its FFT (scipy.fft) on %d host threads; "
                      "setup untimed" % (iters, workload_name(args), cores),
            "single_core": {"value": 1.0 / dt1, "unit": "iter/s", "cores": 1,
                            "sample": "%d timed iterations, one thread"
                                      % max(2, iters // 5)}}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import scipy.fft as sfft
    prob = workload(args)
    cf, Lh, uo = _oracle_setup(prob)
    alpha = uo.alpha_star(cf["V"])
    cores = _host_cores()
    x = np.zeros_like(cf["y"])
    with sfft.set_workers(cores):
        for _ in range(max(args.warmup, 0)):
            x, _ = uo.iterate(cf["V"], cf["y"], Lh, alpha, 1, x0=x, ref_norm=1.0)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            x, _ = uo.iterate(cf["V"], cf["y"], Lh, alpha, 1, x0=x, ref_norm=1.0)
        dt = time.perf_counter() - t0
    value = args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iter/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args),
                   "grid": [args.n] * args.ndim, "tol": args.tol,
                   "step": "one iteration of the FP64 CPU oracle (bounded sample)"},
        "cpu_baseline": {"value": value, "unit": "iter/s", "cores": cores, "kind": "oracle",
                         "sample": "%d timed iterations of Algorithm 1 (FP64 oracle, FFT on "
                                   "%d host threads) on the %s workload"
                                   % (args.steps, cores, workload_name(args))},
        "e2e": {"value": value, "unit": "iter/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
