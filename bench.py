"""Benchmark of the staggered Dslash and even-odd CG path on GB300.

Workload (one GPU): the 32^3 x 8 lattice, smooth links exp(0.3 i H), m = 0.01,
Gaussian source, plain double precision (F64 storage, 18-real links).  One
step is a complete CG solve of M x = b to a true relative residual of 1e-10:
every half-Dslash application, the fused BLAS and reductions, and the
device-side iteration loop, with the inputs resident in HBM.

Printed value: Dslash GFLOP/s sustained over the solve = 570 flop x V/2 sites x
(half-Dslash applications in the solve) / solve time (the paper's 570
flop/site count, Sec. 4.3).  Extra keys report CG time-to-solution, the
standalone Dslash kernel against its roofline, an end-to-end number through
the C ABI with host buffers, and the CPU oracle timed on the host cores.

``--impl reference`` times the CPU oracle on the same workload (bounded
samples: a few CG iterations per step) and prints the same line with
"impl": "reference".

Multi-GPU (torchrun): every rank solves its own right-hand side (independent
problems, weak scaling, no collective on the data path); the step time is the
maximum over ranks.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import lattice_inputs as li  # noqa: E402

METRIC = "Dslash GFLOP/s + HBM roofline frac; CG time-to-solution FP64 vs mixed/multi-RHS"
FLOP_PER_SITE = 570            # Sec. 4.3: per output site of one half-Dslash
WORKLOAD_INDEX = 1             # 32^3 x 8 smooth eps=0.3, m=0.01
TOL = 1e-10
L2_FLUSH_BYTES = 512 << 20     # larger than the 129 MB L2

# algorithmic bytes per output site of a half-Dslash: 8 links read once,
# the input spinor once, the output once (links are each used once per half)
def dslash_bytes_per_site(prec_bytes: int, recon: int) -> int:
    return 8 * recon * prec_bytes + 2 * 6 * prec_bytes


def paper_float_count(n: int = 1) -> int:
    """Floats per site in the paper's model (Sec. 4.3): 6 links x 12 + n x 9 vectors x 6."""
    return 6 * 12 + n * 9 * 6


def paper_arithmetic_intensity(n: int, bytes_per_float: int = 8) -> float:
    """n * 570 / (8 * (6*12 + n*9*6)) flop/byte for FP64 (Sec. 4.3)."""
    return n * FLOP_PER_SITE / (bytes_per_float * paper_float_count(n))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# FP64 FMA rate of GB300 from unit counts and clock: the FP64 pipe issues
# 1/64 of the FP32 rate; 152 SMs x 128 FP32 lanes / 64 x 2 flop x 2.07 GHz.
def fp64_peak_gflops(sm_mhz: float = 2070.0) -> float:
    return 152 * (128 / 64) * 2 * sm_mhz * 1e-3


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- reference

def run_reference(args, ws, rank):
    """The CPU oracle as it stands (single thread), bounded CG samples per step."""
    if rank != 0:
        return 0
    import oracle as orc
    w = li.WORKLOADS[WORKLOAD_INDEX]
    dims, mass = w["dims"], w["mass"]
    U = li.random_links(dims, "smooth", eps=w["eps"], seed=li.workload_seed(WORKLOAD_INDEX, 0))
    b = li.gaussian_half(dims, seed=li.workload_seed(WORKLOAD_INDEX, 1))
    Vh = li.volume(dims) // 2
    iters_per_step = 2

    def step():
        t0 = time.perf_counter()
        _, it, _, _ = orc.cg(dims, U, mass, b, tol=TOL, maxiter=iters_per_step)
        dt = time.perf_counter() - t0
        return dt, 2 * (it + 1)      # two half-Dslashes per M; one more M for the true residual

    for _ in range(args.warmup):
        step()
    tot_t, tot_h = 0.0, 0
    for _ in range(args.steps):
        dt, nh = step()
        tot_t += dt
        tot_h += nh
    gflops = FLOP_PER_SITE * Vh * tot_h / tot_t * 1e-9
    sample = f"oracle CG on {dims}, {iters_per_step} iterations + true residual per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": gflops, "unit": "GFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_t / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w["name"], "dims": list(dims), "mass": mass},
        "cpu_baseline": {"value": gflops, "unit": "GFLOP/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": gflops, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_sample(dims, U, b, mass, Vh, budget_s=12.0):
    """Oracle timed on the host (single thread) on a bounded sample of the workload."""
    import oracle as orc
    t0 = time.perf_counter()
    n_half = 0
    its = 0
    while time.perf_counter() - t0 < budget_s:
        _, it, _, _ = orc.cg(dims, U, mass, b, tol=TOL, maxiter=2)
        n_half += 2 * (it + 1)
        its += 1
    dt = time.perf_counter() - t0
    return {"value": FLOP_PER_SITE * Vh * n_half / dt * 1e-9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
            "sample": f"{its} oracle CG runs of 2 iterations + true residual on {dims} ({n_half} half-Dslashes, "
                      f"{dt:.1f} s)"}


# ---------------------------------------------------------------- ours

def profile_kernel(args, stag, torch):
    """A few launches of one operator on the workload, nothing timed (an ncu target)."""
    name = args.profile_kernel
    kern, _, dtxt = name.partition("@")
    parts = kern.split("_")
    prec = {"f64": stag.F64, "f32": stag.F32, "f16": stag.F16}[parts[1]]
    recon = int(parts[2])
    w = li.WORKLOADS[WORKLOAD_INDEX]
    dims = tuple(int(v) for v in dtxt.split("x")) if dtxt else w["dims"]
    U = li.random_links(dims, "smooth", eps=w["eps"], seed=li.workload_seed(WORKLOAD_INDEX, 0))
    ctx = stag.Context(dims)
    ctx.upload_gauge(torch.from_numpy(U).cuda())
    psi = torch.from_numpy(li.gaussian_half(dims, seed=99)).cuda()
    out = ctx.new_half()
    for _ in range(args.warmup + args.steps):
        ctx.dslash_eo(out, psi, prec, recon)
    torch.cuda.synchronize()
    print(json.dumps({"profile_kernel": name, "workload": w["name"], "launches": args.warmup + args.steps}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--use-graph", type=int, default=1,
                    help="1: device-side loop in one CUDA graph; 0: host-driven loop (per-kernel profiling)")
    ap.add_argument("--profile-kernel", default=None,
                    help="only run a few launches of one kernel on the workload (for ncu): "
                         "dslash_f64_18, dslash_f32_12, dslash_f16_12, ...; optional @LXxLYxLZxLT lattice")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2502_03249_gb300 as stag
    stag.load()
    if args.profile_kernel:
        return profile_kernel(args, stag, torch)

    w = li.WORKLOADS[WORKLOAD_INDEX]
    dims, mass = w["dims"], w["mass"]
    Vh = li.volume(dims) // 2
    U = li.random_links(dims, "smooth", eps=w["eps"], seed=li.workload_seed(WORKLOAD_INDEX, 0))
    b_np = li.gaussian_half(dims, seed=li.workload_seed(WORKLOAD_INDEX, 1) + 7919 * rank)
    dev = torch.device("cuda", local)
    ctx = stag.Context(dims)
    ctx.upload_gauge(torch.from_numpy(U).to(dev))
    b = torch.from_numpy(b_np).to(dev)
    x = ctx.new_half()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            dist.barrier()

    ug = args.use_graph
    for _ in range(args.warmup):
        st = ctx.cg_solve(x, b, mass, tol=TOL, use_graph=ug)
    torch.cuda.synchronize()

    # ---- timed region: K complete solves, L2 flushed between them
    times, stats = [], []
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = ctx.cg_solve(x, b, mass, tol=TOL, use_graph=ug)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            stats.append(st)
    torch.cuda.synchronize()
    barrier()
    t_sum = sum(times)
    if ws > 1:
        tt = torch.tensor([t_sum], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_sum = float(tt.item())
    ms_per_step = t_sum / args.steps
    n_half = [2 * (s["iters"] + s["restarts"] + 1) for s in stats]
    half_per_step = statistics.mean(n_half)
    value = ws * FLOP_PER_SITE * Vh * half_per_step / (ms_per_step * 1e-3) * 1e-9
    launches = sum(1 + 4 * s["iters"] + 2 * (s["restarts"] + 1) + s["restarts"] for s in stats)

    # ---- standalone Dslash kernel (F64/18) for the roofline: events per launch, L2 flushed
    out = ctx.new_half()
    psi = torch.from_numpy(li.gaussian_half(dims, seed=99)).to(dev)
    for _ in range(5):
        ctx.dslash_eo(out, psi)
    ks = []
    for _ in range(30):
        flush.fill_(2.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.dslash_eo(out, psi)
        e1.record(stream)
        e1.synchronize()
        ks.append(e0.elapsed_time(e1))
    k_ms = statistics.mean(ks)
    k_bytes = dslash_bytes_per_site(8, 18) * Vh
    k_gbs = k_bytes / (k_ms * 1e-3) * 1e-9
    k_gflops = FLOP_PER_SITE * Vh / (k_ms * 1e-3) * 1e-9
    peaks, peak_kind = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    clocks = clk.summary()
    fp64_peak = fp64_peak_gflops()

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region
    b_host = torch.from_numpy(b_np).pin_memory()
    x_host = torch.empty_like(b_host).pin_memory()
    xd = ctx.new_half()
    bd = torch.empty_like(xd)
    e2e_t = []
    e2e_half = []
    for _ in range(max(2, args.steps // 2)):
        flush.fill_(3.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bd.copy_(b_host, non_blocking=True)
        st = ctx.cg_solve(xd, bd, mass, tol=TOL)
        x_host.copy_(xd, non_blocking=True)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
        e2e_half.append(2 * (st["iters"] + st["restarts"] + 1))
    e2e_val = FLOP_PER_SITE * Vh * statistics.mean(e2e_half) / statistics.mean(e2e_t) * 1e-9

    # ---- mixed precision on the same workload: time-to-solution at the same true residual
    mixed = {}
    for name, prec, recon in (("f32_12", stag.F32, 12), ("f16_12", stag.F16, 12)):
        xm = ctx.new_half()
        for _ in range(2):
            ctx.cg_solve_mixed(xm, b, mass, tol=TOL, inner_prec=prec, inner_recon=recon, use_graph=ug)
        tm = []
        for _ in range(3):
            flush.fill_(4.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sm = ctx.cg_solve_mixed(xm, b, mass, tol=TOL, inner_prec=prec, inner_recon=recon, use_graph=ug)
            e1.record(stream)
            e1.synchronize()
            tm.append(e0.elapsed_time(e1))
        mixed[name] = {"time_to_solution_ms": statistics.median(tm), "iters": sm["iters"],
                       "reliable_updates": sm["reliable_updates"], "true_rel_residual": sm["true_rel_residual"],
                       "speedup_vs_f64": ms_per_step / statistics.median(tm)}

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return 0

    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline_sample(dims, U, b_np, mass, Vh)

    last = stats[-1]
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "GFLOP/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {
            "workload": w["name"] + ", double-precision CG to true residual 1e-10 (one solve per step)",
            "dims": list(dims), "mass": mass, "links": "exp(0.3 i H), 18-real F64", "tol": TOL,
            "l2": "flushed (512 MB write) before every step; working set 151 MB links + 6 MB per vector",
            "value_definition": "570 flop x V/2 x half-Dslash applications per solve / solve time",
        },
        "cg": {"time_to_solution_ms": ms_per_step, "iters": last["iters"], "restarts": last["restarts"],
               "true_rel_residual": last["true_rel_residual"], "half_dslash_per_solve": half_per_step},
        "roofline": {
            "kernel": "k_dslash<F64/18> (stag_dslash_eo)", "bound": "alu",
            "achieved": k_gflops, "peak": fp64_peak, "unit": "GFLOP/s", "frac": k_gflops / fp64_peak,
            "traffic": None,
            "peak_source": "FP64 FMA rate from unit counts and max clock (152 SM x 2 DFMA/clk x 2.07 GHz)",
            "hbm": {"achieved_gbs": k_gbs, "peak_gbs": hbm, "frac": k_gbs / hbm, "peak_source": peak_kind,
                    "algorithmic_bytes_per_site": dslash_bytes_per_site(8, 18)},
            "kernel_ms": k_ms,
        },
        "e2e": {"value": e2e_val, "unit": "GFLOP/s", "h2d_bytes_per_step": int(b_host.numel() * 16),
                "d2h_bytes_per_step": int(x_host.numel() * 16), "seconds_per_step": statistics.mean(e2e_t)},
        "mixed": mixed,
        "gpu_launches": launches,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
