"""Benchmark of the staggered Dslash and even-odd CG path on GB300.

Headline step (one GPU): the 48^3 x 12 lattice, smooth links exp(0.2 i H),
m = 0.002, Gaussian source.  One step is a complete double-precision CG solve
of M x = b in IEEE double arithmetic (double links, vectors and FP64
operations: the paper's "DP" CG, Sec. 4.2 and Table 1) to a true relative
residual of 1e-10 -- every half-Dslash application, the BLAS and reductions,
the device-side iteration loop -- with the inputs resident in HBM and L2
flushed before every step.

Printed value: Dslash GFLOP/s sustained over the solve = 570 flop x V/2 sites
x (half-Dslash applications in the solve) / solve time (the paper's 570
flop/site count, Sec. 4.3); ms_per_step is the CG time-to-solution.  Beside it,
on the same workload and source: the double-float CG (double storage, FP32-pipe
arithmetic), the same in temporal gauge, and the mixed-precision solves (float
and half 12-real inner iterations with double reliable updates), each with its
speed-up over the IEEE solve; the operator kernels against their rooflines (the
IEEE operator against the FP64 FMA peak and against HBM); an end-to-end number
through the C ABI with host buffers; batched multi-RHS, multi-shift, force and
32^3 x 8 sections; the CPU oracle timed on the host cores.

``--impl reference`` times the CPU oracle (its OpenMP build, every host core)
on the same workload (bounded samples: a few CG iterations per step) and prints
the same line with "impl": "reference".

Multi-GPU (torchrun): every rank solves its own right-hand side (independent
problems, weak scaling, no collective on the data path); the step time is the
maximum over ranks.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import lattice_inputs as li  # noqa: E402

METRIC = "Dslash GFLOP/s + HBM roofline frac; CG time-to-solution FP64 vs mixed/multi-RHS"
FLOP_PER_SITE = 570            # Sec. 4.3: per output site of one half-Dslash
WORKLOAD_INDEX = 2             # 48^3 x 12 smooth eps=0.2, m=0.002
TOL = 1e-10
L2_FLUSH_BYTES = 512 << 20     # larger than the 129 MB L2
SHIFTS12 = [10.0 ** (-5 + 5 * i / 11) for i in range(12)]
F64_IEEE, F64X = 0, 3


# algorithmic bytes per output site of a half-Dslash: 8 links read once,
# the input spinor once, the output once (links are each used once per half)
def dslash_bytes_per_site(prec_bytes: int, recon: int) -> int:
    return 8 * recon * prec_bytes + 2 * 6 * prec_bytes


# the same in temporal gauge (Sec. 4.3): the 6 spatial links, and a time link
# only where it is not the identity (the forward one on the last slice, the
# backward one on slice 0: 2 / Lt links per site on average)
def dslash_bytes_per_site_tg(prec_bytes: int, recon: int, lt: int) -> float:
    return (6 + 2.0 / lt) * recon * prec_bytes + 2 * 6 * prec_bytes


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


def load_traffic():
    """DRAM bytes per launch of the profiled kernels (ncu captures, profiles/traffic.json)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


# FP64 FMA rate of GB300 from unit counts and clock: the FP64 pipe issues
# 1/64 of the FP32 rate; 152 SMs x 128 FP32 lanes / 64 x 2 flop x 2.07 GHz.
def fp64_peak_gflops(sm_mhz: float = 2070.0) -> float:
    return 152 * (128 / 64) * 2 * sm_mhz * 1e-3


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region.

    A reader thread timestamps every sample; entering waits (up to 10 s) for
    the first sample so that the sampler is running when the timed region
    starts, and only samples taken between entering and leaving (plus one
    interval) are summarised."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 50

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.samples = []          # (perf_counter time, csv line)
        self.lines = []

    def _read(self):
        for ln in self.proc.stdout:
            if ln.strip():
                self.samples.append((time.perf_counter(), ln))

    def __enter__(self):
        import threading
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        if self.proc is not None:
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t_end = time.perf_counter() + 10.0
            while not self.samples and time.perf_counter() < t_end and self.proc.poll() is None:
                time.sleep(0.01)
        self.t0 = time.perf_counter()
        return self

    def __exit__(self, *exc):
        self.t1 = time.perf_counter()
        if self.proc is not None:
            time.sleep(self.INTERVAL_MS * 1e-3)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
                self.proc.wait()
            self.thread.join(timeout=5)
        hi = self.t1 + self.INTERVAL_MS * 1e-3
        self.lines = [ln for t, ln in self.samples if self.t0 <= t <= hi]

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


def max_over_ranks(value: float, ws: int, device=None) -> float:
    """Maximum of a per-rank time over all ranks (the timing harness's only collective)."""
    if ws <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(ws: int, vh: int, half_dslash_per_step: float, ms_per_step: float) -> float:
    """Whole-job Dslash GFLOP/s: every rank solves its own system, so the units of
    work are summed over ranks and divided by the slowest rank's time."""
    return ws * FLOP_PER_SITE * vh * half_dslash_per_step / (ms_per_step * 1e-3) * 1e-9


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- reference

def run_reference(args, ws, rank):
    """The CPU oracle as it stands (its OpenMP build on every host core),
    bounded CG samples per step on the headline workload."""
    if rank != 0:
        return 0
    import oracle as orc
    w = li.WORKLOADS[WORKLOAD_INDEX]
    dims, mass = w["dims"], w["mass"]
    U = li.random_links(dims, "smooth", eps=w["eps"], seed=li.workload_seed(WORKLOAD_INDEX, 0))
    b = li.gaussian_half(dims, seed=li.workload_seed(WORKLOAD_INDEX, 1))
    Vh = li.volume(dims) // 2
    iters_per_step = 2

    with orc.threads():
        cores = orc.num_threads()

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
    sample = (f"oracle CG on {dims}, {iters_per_step} iterations + true residual per step, OpenMP build on "
              f"{cores} host threads ({cpu_model()})")
    line = {
        "impl": "reference", "metric": METRIC, "value": gflops, "unit": "GFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_t / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": headline_config(w),
        "cpu_baseline": {"value": gflops, "unit": "GFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": gflops, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part", "hardware")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def headline_config(w):
    """The benchmark step's workload, the same dict in both arms' lines."""
    return {
        "workload": w["name"] + ", IEEE double CG to true residual 1e-10 (one solve per step)",
        "dims": list(w["dims"]), "mass": w["mass"], "links": f"exp({w['eps']} i H), 18-real double", "tol": TOL,
        "arithmetic": "IEEE double (links, vectors, operator, BLAS, reductions)",
        "l2": "GPU arm: flushed (512 MB write, then 512 MB read) before every step; working set 764 MB links "
              "+ 32 MB per vector (larger than L2)",
        "value_definition": "570 flop x V/2 x half-Dslash applications per solve / solve time",
    }


def cpu_baseline_sample(dims, U, b, mass, Vh, budget_s=12.0):
    """Oracle timed on the host cores (its OpenMP build) on a bounded sample of
    the workload: whole CG runs of 2 iterations plus the true residual."""
    import oracle as orc
    with orc.threads():
        cores = orc.num_threads()
        t0 = time.perf_counter()
        n_half = 0
        its = 0
        while time.perf_counter() - t0 < budget_s:
            _, it, _, _ = orc.cg(dims, U, mass, b, tol=TOL, maxiter=2)
            n_half += 2 * (it + 1)
            its += 1
        dt = time.perf_counter() - t0
    return {"value": FLOP_PER_SITE * Vh * n_half / dt * 1e-9, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
            "sample": f"{its} oracle CG runs of 2 iterations + true residual on {dims} ({n_half} half-Dslashes, "
                      f"{dt:.1f} s), OpenMP build on {cores} threads ({cpu_model()})"}


# ---------------------------------------------------------------- helpers

CG_GRAPH_UNROLL = 4     # CG iterations per body of the solver graph's while loop
CG_CHECK_EVERY = 25     # host-driven loop: iterations between convergence reads


def cg_df_dir(vh, l2_bytes):
    """Whether the double-float CG applies p = r + beta p inside its operator
    passes (three launches per iteration): the library's rule, five 48-byte
    vectors per site within half of L2, unless STAG_CG_DIR forces it."""
    e = os.environ.get("STAG_CG_DIR", "")
    if e[:1] in ("0", "1"):
        return e[:1] == "1"
    return 5 * 48 * vh <= 0.5 * l2_bytes


def cg_kernel_launches(st, use_graph, arith=0, df_dir=True):
    """Kernels one double-precision CG solve launches: the normalisation of b
    (largest-magnitude pass, exponent, scaled copy), the start kernel, four per
    iteration slot (whole graph bodies, or whole host-loop batches; three when
    the double-float solver applies p = r + beta p inside its operator passes,
    df_dir), the two true-residual kernels per pass, one restart kernel per
    restart and the scaled copy of the solution.  Exact when the solve needed
    no restart (each pass's iterations are not reported separately)."""
    per = CG_GRAPH_UNROLL if use_graph else CG_CHECK_EVERY
    passes = st["restarts"] + 1
    slots = per * max(passes, math.ceil(max(st["iters"], 1) / per))
    per_iter = 3 if (arith == F64X and df_dir) else 4
    return 3 + 1 + per_iter * slots + 2 * passes + st["restarts"] + 1


class L2Flush:
    """Evict L2 before a timed call: write a buffer larger than L2, then read a
    second one, so that L2 holds clean lines of the second buffer.  (Without the
    read, the timed kernel would pay for writing back up to 129 MB of dirty
    lines left by the write, which no kernel of the path produced.)"""

    def __init__(self, torch, dev):
        self.torch = torch
        self.w = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        self.r = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        self.o = torch.zeros((), dtype=torch.float32, device=dev)

    def __call__(self, v=1.0):
        self.w.fill_(v)
        self.torch.sum(self.r, 0, out=self.o)


class Timer:
    """CUDA-event timing of a callable on the current stream, L2 flushed before each call."""

    def __init__(self, torch, flush):
        self.torch = torch
        self.flush = flush

    def __call__(self, fn, reps=3, warm=1):
        torch = self.torch
        for _ in range(warm):
            fn()
        out, ts = None, []
        stream = torch.cuda.current_stream()
        for _ in range(reps):
            self.flush(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts), out


def dslash_kernel_entry(timer, ctx, psi, out, prec, recon, vh, hbm, tg=False):
    """The bare operator kernel (internal storage, no conversions), one launch per timing.
    tg: on the temporal-gauge links, identity time links skipped (GFLOP/s then
    counts the paper's 570 flop per site although the skipped hops do less)."""
    import paper_2502_03249_gb300 as stag
    ctx.set_operator_links(stag.LINKS_TEMPORAL if tg else stag.LINKS_UPLOADED)
    ctx.dslash_prepare(psi, prec)
    ms, _ = timer(lambda: ctx.dslash_repeat(prec, recon, 1), reps=20, warm=3)
    ctx.set_operator_links(stag.LINKS_UPLOADED)
    pb = {0: 8, 3: 8, 1: 4, 2: 2}[prec]
    lt = ctx.dims[3]
    per_site = (dslash_bytes_per_site_tg(pb, recon, lt) if tg else dslash_bytes_per_site(pb, recon)) + \
        (8 if prec == 2 else 0)
    gbs = per_site * vh / (ms * 1e-3) * 1e-9
    return {"ms": ms, "gflops": FLOP_PER_SITE * vh / (ms * 1e-3) * 1e-9, "achieved_gbs": gbs,
            "frac_of_hbm": gbs / hbm, "algorithmic_bytes_per_site": per_site,
            "links": "temporal gauge (6 + 2/Lt link reads per site)" if tg else "as uploaded (8 per site)"}


def profile_kernel(args, stag, torch):
    """A few launches of one operator on the workload, nothing timed (an ncu target)."""
    name = args.profile_kernel
    kern, _, dtxt = name.partition("@")
    parts = kern.split("_")
    w = li.WORKLOADS[WORKLOAD_INDEX]
    dims = tuple(int(v) for v in dtxt.split("x")) if dtxt else w["dims"]
    if parts[0] in ("multi", "multishift", "mixed", "force") or (parts[0] == "dslash" and parts[1] == "all"):
        U = None   # these modes generate their inputs on the device
    else:
        U = li.random_links(dims, "smooth", eps=w["eps"], seed=li.workload_seed(WORKLOAD_INDEX, 0))
        ctx = stag.Context(dims)
        ctx.upload_gauge(torch.from_numpy(U).cuda())
    if parts[0] in ("multi", "multishift"):
        # the 32^3 x 16 batched (16 RHS) or multi-shift (12 shifts) solve, host-driven
        w3 = li.WORKLOADS[3]
        dims3 = tuple(int(v) for v in dtxt.split("x")) if dtxt else w3["dims"]
        ctx = stag.Context(dims3)
        ctx.upload_gauge(li.random_links_torch(dims3, "smooth", w3["eps"], seed=li.workload_seed(3, 0)))
        B = li.gaussian_half_torch(dims3, seed=li.workload_seed(3, 1), nvec=16)
        prec = {"f32": stag.F32, "f16": stag.F16}[parts[1]]
        for _ in range(args.warmup + args.steps):
            if parts[0] == "multi":
                X = ctx.new_half(16)
                ctx.cg_solve_multi(X, B, w3["mass"], tol=TOL, inner_prec=prec, inner_recon=int(parts[2]), use_graph=0)
            else:
                X = ctx.new_half(12)
                ctx.cg_solve_multishift(X, B[0].contiguous(), SHIFTS12, w3["mass"], tol=TOL, inner_prec=prec,
                                        inner_recon=int(parts[2]), use_graph=0)
        torch.cuda.synchronize()
        print(json.dumps({"profile_kernel": name, "workload": w3["name"], "solves": args.warmup + args.steps}))
        return 0
    if parts[0] == "mixed":
        # the 48^3 x 12 mixed-precision solve (inner F32 or F16, 12-real), host-driven
        w2 = li.WORKLOADS[2]
        dims2 = tuple(int(v) for v in dtxt.split("x")) if dtxt else w2["dims"]
        ctx = stag.Context(dims2)
        ctx.upload_gauge(li.random_links_torch(dims2, "smooth", w2["eps"], seed=li.workload_seed(2, 0)))
        b = li.gaussian_half_torch(dims2, seed=li.workload_seed(2, 1))
        x = ctx.new_half()
        prec = {"f32": stag.F32, "f16": stag.F16}[parts[1]]
        tg = 1 if len(parts) > 3 and parts[3] == "tg" else 0   # mixed_<prec>_12_tg: in temporal gauge
        for _ in range(args.warmup + args.steps):
            ctx.cg_solve_mixed(x, b, w2["mass"], tol=TOL, inner_prec=prec, inner_recon=int(parts[2]), use_graph=0,
                               temporal_gauge=tg)
        torch.cuda.synchronize()
        print(json.dumps({"profile_kernel": name, "workload": w2["name"], "solves": args.warmup + args.steps}))
        return 0
    if parts[0] == "cg":
        # whole solves, host-driven (ncu does not see the kernels of graphs with conditional nodes);
        # cg_f64x_tg: in temporal gauge
        arith = {"f64": F64_IEEE, "f64x": F64X}[parts[1]]
        tg = 1 if len(parts) > 2 and parts[2] == "tg" else 0
        b = torch.from_numpy(li.gaussian_half(dims, seed=li.workload_seed(WORKLOAD_INDEX, 1))).cuda()
        x = ctx.new_half()
        for _ in range(args.warmup + args.steps):
            ctx.cg_solve(x, b, w["mass"], tol=TOL, use_graph=0, f64_arith=arith, temporal_gauge=tg)
        torch.cuda.synchronize()
        print(json.dumps({"profile_kernel": name, "workload": w["name"], "solves": args.warmup + args.steps}))
        return 0
    if parts[0] == "dslash" and parts[1] == "all":
        # one bare operator launch per storage (IEEE double, double-float, float/12,
        # half/12) on torch-generated inputs of the headline recipe, after
        # warm-up launches of each
        ctx = stag.Context(dims)
        ctx.upload_gauge(li.random_links_torch(dims, "smooth", w["eps"], seed=li.workload_seed(WORKLOAD_INDEX, 0)))
        psi = li.gaussian_half_torch(dims, seed=99)
        for prec, recon in ((stag.F64, 18), (stag.F64X, 18), (stag.F32, 12), (stag.F16, 12)):
            ctx.dslash_prepare(psi, prec)
            for _ in range(args.warmup):
                ctx.dslash_repeat(prec, recon, 1)
        torch.cuda.synchronize()
        for prec, recon in ((stag.F64, 18), (stag.F64X, 18), (stag.F32, 12), (stag.F16, 12)):
            ctx.dslash_prepare(psi, prec)
            ctx.dslash_repeat(prec, recon, 1)
        torch.cuda.synchronize()
        print(json.dumps({"profile_kernel": name, "dims": list(dims), "launches": 4 * (args.warmup + 1)}))
        return 0
    if parts[0] == "force":
        # the projected force on 32^3 x 16 (64^3 x 16 recipe, eps = 0.3, m = 0.01): X from a solve,
        # then warm-up and one measured stag_fermion_force call (P only)
        w5 = li.WORKLOADS[5]
        dimsf = tuple(int(v) for v in dtxt.split("x")) if dtxt else (32, 32, 32, 16)
        ctx = stag.Context(dimsf)
        U5 = li.random_links_torch(dimsf, "smooth", w5["eps"], seed=li.workload_seed(5, 0))
        ctx.upload_gauge(U5)
        phi = li.gaussian_half_torch(dimsf, seed=li.workload_seed(5, 1))
        _, X, _ = ctx.fermion_action(phi, w5["mass"], tol=TOL)
        P = torch.empty_like(U5)
        for _ in range(args.warmup + args.steps):
            ctx.fermion_force(X, P=P)
        torch.cuda.synchronize()
        print(json.dumps({"profile_kernel": name, "dims": list(dimsf), "calls": args.warmup + args.steps}))
        return 0
    prec = {"f64": stag.F64, "f32": stag.F32, "f16": stag.F16, "f64x": stag.F64X}[parts[1]]
    recon = int(parts[2])
    psi = torch.from_numpy(li.gaussian_half(dims, seed=99)).cuda()
    # dslash_<prec>_<recon>_tg: on the temporal-gauge links (identity time links skipped)
    if len(parts) > 3 and parts[3] == "tg":
        ctx.set_operator_links(stag.LINKS_TEMPORAL)
    # the bare kernel on the precision's internal storage, as the benchmark times it
    ctx.dslash_prepare(psi, prec)
    for _ in range(args.warmup + args.steps):
        ctx.dslash_repeat(prec, recon, 1)
    torch.cuda.synchronize()
    print(json.dumps({"profile_kernel": name, "workload": w["name"], "launches": args.warmup + args.steps}))
    return 0


MULTI_CONFIGS = [(1, 1), (1, 2), (1, 4), (1, 8), (2, 1), (2, 2), (4, 1), (2, 4), (4, 2), (8, 1), (2, 8), (4, 4),
                 (8, 2), (16, 1)]   # (G warp groups sharing a link tile, NBT right-hand sides per thread)


def sweep_multi(args, stag, torch):
    """Every multi-vector configuration on the paper's Table 2 lattice recipe
    (smooth links eps = 0.3): TFLOP/s (570 flop per site per vector) and the
    fraction of the HBM roof of the compulsory bytes, (384 + 48 n) / n B per
    site-vector for float/12 and (192 + 32 n) / n for half/12."""
    dims = tuple(int(v) for v in args.sweep_multi.split("x"))
    Vh = li.volume(dims) // 2
    hbm = float(load_peaks()[0]["hbm_gbs"])
    ctx = stag.Context(dims)
    ctx.upload_gauge(li.random_links_torch(dims, "smooth", 0.3, seed=li.workload_seed(6, 0)))
    psi = li.gaussian_half_torch(dims, seed=li.workload_seed(6, 1), nvec=16)
    timer = Timer(torch, L2Flush(torch, torch.device("cuda", torch.cuda.current_device())))
    for label, prec, lb, sb in (("f32_12", stag.F32, 384, 48), ("f16_12", stag.F16, 192, 32)):
        for n in (1, 2, 4, 8, 16):
            ctx.dslash_prepare_multi(psi[:n].contiguous(), prec)
            cap = 1
            while cap < n:
                cap *= 2
            roof = hbm * 1e9 / ((lb + sb * n) / n) * FLOP_PER_SITE * 1e-12
            row = {}
            for G, N in MULTI_CONFIGS:
                if G * N > cap:
                    continue
                ms, _ = timer(lambda: ctx.dslash_repeat_multi(prec, 12, (G << 8) | N, 1), reps=7, warm=2)
                tf = FLOP_PER_SITE * Vh * n / (ms * 1e-3) * 1e-12
                row[f"{G}x{N}"] = {"us": round(ms * 1e3, 1), "tflops": round(tf, 2), "frac": round(tf / roof, 3)}
            ctx.dslash_repeat_multi(prec, 12, 0, 1)
            best = max(row.items(), key=lambda kv: kv[1]["tflops"])
            print(json.dumps({"storage": label, "dims": list(dims), "n": n, "roof_tflops": round(roof, 2),
                              "autotuned_block": ctx.last_rhs_block(), "best": best, "configs": row}), flush=True)
    return 0


def half_dslash(st):
    # two half-Dslashes per M application, one more M per true-residual check
    return 2 * (st["iters"] + st["restarts"] + 1)


# ---------------------------------------------------------------- sections

def section_32c8(stag, torch, timer, hbm):
    """32^3 x 8, eps = 0.3, m = 0.01: the double CG in both arithmetics and in
    temporal gauge, the mixed solves, and the operator kernels (L2-assisted:
    the 151 MB of double links barely exceed L2)."""
    w = li.WORKLOADS[1]
    dims, mass = w["dims"], w["mass"]
    ctx = stag.Context(dims)
    ctx.upload_gauge(li.random_links_torch(dims, "smooth", w["eps"], seed=li.workload_seed(1, 0)))
    b = li.gaussian_half_torch(dims, seed=li.workload_seed(1, 1))
    x = ctx.new_half()
    vh = ctx.Vh
    res = {"workload": w["name"] + " (inputs from the torch generator)"}
    ms_i, st = timer(lambda: ctx.cg_solve(x, b, mass, tol=TOL, f64_arith=F64_IEEE), reps=3)
    res["cg_ieee_f64"] = {"time_to_solution_ms": ms_i, "iters": st["iters"],
                          "true_rel_residual": st["true_rel_residual"],
                          "gflops": FLOP_PER_SITE * vh * half_dslash(st) / (ms_i * 1e-3) * 1e-9}
    ms, st = timer(lambda: ctx.cg_solve(x, b, mass, tol=TOL, f64_arith=F64X), reps=3)
    res["cg_f64x"] = {"time_to_solution_ms": ms, "iters": st["iters"], "true_rel_residual": st["true_rel_residual"],
                      "speedup_vs_cg_ieee_f64": ms_i / ms}
    ctx.cg_solve(x, b, mass, tol=TOL, temporal_gauge=1)   # builds the transform once
    m, s_ = timer(lambda: ctx.cg_solve(x, b, mass, tol=TOL, temporal_gauge=1), reps=3)
    res["cg_f64x_temporal_gauge"] = {"time_to_solution_ms": m, "iters": s_["iters"],
                                     "true_rel_residual": s_["true_rel_residual"], "speedup_vs_cg_ieee_f64": ms_i / m}
    for name, prec in (("mixed_f32_12", stag.F32), ("mixed_f16_12", stag.F16)):
        m, s_ = timer(lambda: ctx.cg_solve_mixed(x, b, mass, tol=TOL, inner_prec=prec, inner_recon=12), reps=3)
        res[name] = {"time_to_solution_ms": m, "iters": s_["iters"], "reliable_updates": s_["reliable_updates"],
                     "true_rel_residual": s_["true_rel_residual"], "speedup_vs_cg_ieee_f64": ms_i / m}
    psi = li.gaussian_half_torch(dims, seed=99)
    out = ctx.new_half()
    res["dslash"] = {name: dslash_kernel_entry(timer, ctx, psi, out, p, r, vh, hbm)
                     for name, p, r in (("f64x_18", F64X, 18), ("f64_18", F64_IEEE, 18), ("f32_12", stag.F32, 12),
                                        ("f16_12", stag.F16, 12))}
    ctx.close()
    return res


def section_32c16(stag, torch, timer):
    """32^3 x 16, eps = 0.3, m = 0.005: 16 RHS batched, 12 shifts multi-shift, against sequential solves."""
    w = li.WORKLOADS[3]
    dims, mass = w["dims"], w["mass"]
    ctx = stag.Context(dims)
    ctx.upload_gauge(li.random_links_torch(dims, "smooth", w["eps"], seed=li.workload_seed(3, 0)))
    B = li.gaussian_half_torch(dims, seed=li.workload_seed(3, 1), nvec=16)
    X = ctx.new_half(16)
    res = {"workload": w["name"] + " (inputs from the torch generator)"}
    ms_b, st = timer(lambda: ctx.cg_solve_multi(X, B, mass, tol=TOL, inner_prec=stag.F32, inner_recon=12), reps=2)
    res["batched_16rhs_f32_12"] = {"time_to_solution_ms": ms_b, "rhs_block": ctx.last_rhs_block(),
                                   "max_iters": max(s["iters"] for s in st),
                                   "max_true_rel_residual": max(s["true_rel_residual"] for s in st)}
    ms_t, st = timer(lambda: ctx.cg_solve_multi(X, B, mass, tol=TOL, inner_prec=stag.F32, inner_recon=12,
                                                temporal_gauge=1), reps=2)
    res["batched_16rhs_f32_12_temporal_gauge"] = {"time_to_solution_ms": ms_t, "rhs_block": ctx.last_rhs_block(),
                                                  "max_iters": max(s["iters"] for s in st),
                                                  "max_true_rel_residual": max(s["true_rel_residual"] for s in st)}
    xs = ctx.new_half()

    def seq_f64():
        return [ctx.cg_solve(xs, B[k], mass, tol=TOL) for k in range(16)]

    ms_s, _ = timer(seq_f64, reps=1)
    res["sequential_16_cg_f64x_ms"] = ms_s
    res["batched_speedup_vs_sequential_f64x"] = ms_s / ms_b
    b = B[0].contiguous()
    Xs = ctx.new_half(12)
    ms_m, st = timer(lambda: ctx.cg_solve_multishift(Xs, b, SHIFTS12, mass, tol=TOL), reps=2)
    res["multishift_12"] = {"time_to_solution_ms": ms_m, "krylov_iters": st[0]["restarts"],
                            "max_true_rel_residual": max(s["true_rel_residual"] for s in st)}
    ms_mt, st = timer(lambda: ctx.cg_solve_multishift(Xs, b, SHIFTS12, mass, tol=TOL, temporal_gauge=1), reps=2)
    res["multishift_12_temporal_gauge"] = {"time_to_solution_ms": ms_mt, "krylov_iters": st[0]["restarts"],
                                           "max_true_rel_residual": max(s["true_rel_residual"] for s in st)}

    def seq_shifted():
        return [ctx.cg_solve_shifted(xs, b, mass, s, tol=TOL) for s in SHIFTS12]

    ms_q, _ = timer(seq_shifted, reps=1)
    res["sequential_12_shifted_cg_f64x_ms"] = ms_q
    res["multishift_speedup_vs_sequential_f64x"] = ms_q / ms_m
    ctx.close()
    return res


# The paper's own tables (A100, OpenCL; context, not targets)
PAPER_TABLE2_A100 = {1: (2.244, 1.245), 2: (2.532, 1.530), 3: (2.953, 1.929), 4: (3.205, 2.199), 6: (3.090, 2.039),
                     8: (3.006, 2.026), 10: (3.439, 1.693), 12: (3.196, 2.055), 14: (3.091, 1.562),
                     16: (3.045, 2.122)}   # NMULTI: (FP32, FP64) TFLOP/s, 32^4
PAPER_TABLE1_A100_GBS = 1351.0             # CG update routine, FP64, 48^4 (OpenCL; CUDA backend 1317)


def section_paper_tables(stag, torch, timer, hbm):
    """The paper's Table 2 (Dslash TFLOP/s against NMULTI on 32^4) and Table 1
    (bandwidth of the double-precision CG update on 48^4), measured here on the
    same lattices: the multi-vector operator on internal storage, one launch per
    CUDA-event pair with L2 flushed before it; the update kernel back to back
    on vectors 4 x 48 B/site (> L2)."""
    res = {}
    w6 = li.WORKLOADS[6]
    dims = w6["dims"]
    Vh = li.volume(dims) // 2
    ctx = stag.Context(dims)
    ctx.upload_gauge(li.random_links_torch(dims, w6["links"], w6["eps"], seed=li.workload_seed(6, 0)))
    psi = li.gaussian_half_torch(dims, seed=li.workload_seed(6, 1), nvec=16)
    scan = {}
    for label, prec, recon in (("f32_12", stag.F32, 12), ("f32_12_temporal_gauge", stag.F32, 12),
                               ("f16_12", stag.F16, 12), ("f64x_18", stag.F64X, 18), ("f64_12", stag.F64, 12)):
        ctx.set_operator_links(stag.LINKS_TEMPORAL if label.endswith("temporal_gauge") else stag.LINKS_UPLOADED)
        row, blocks = {}, {}
        for n in sorted(PAPER_TABLE2_A100):
            ctx.dslash_prepare_multi(psi[:n].contiguous(), prec)
            ctx.dslash_repeat_multi(prec, recon, 0, 1)      # the autotuner picks the configuration (cached)
            blocks[n] = ctx.last_rhs_block()
            # timed in the tuned configuration (rhs_block 0 reuses the cached
            # decision; a block size alone would not name the link-tile split)
            ms, _ = timer(lambda: ctx.dslash_repeat_multi(prec, recon, 0, 1), reps=5, warm=2)
            row[n] = FLOP_PER_SITE * Vh * n / (ms * 1e-3) * 1e-12
        scan[label] = {"tflops_by_nmulti": row, "rhs_block": blocks, "best": max(row.values())}
    ctx.set_operator_links(stag.LINKS_UPLOADED)
    res["nmulti_32x4"] = {"unit": "TFLOP/s (570 flop per site per vector)", "scan": scan,
                          "paper_a100_fp32_fp64": PAPER_TABLE2_A100,
                          "note": "n vectors per launch, each link loaded once per block of them (the autotuner's "
                                  "choice of the link-tile split); the paper's Table 2 uses 12-real links in "
                                  "temporal gauge (6 links read per site): the *_temporal_gauge row; the others "
                                  "read 8 links per site"}
    ctx.close()
    dims = li.WORKLOADS[7]["dims"]
    Vh = li.volume(dims) // 2
    ctx = stag.Context(dims)
    upd = {}
    for label, arith in (("f64_ieee", F64_IEEE), ("f64x", F64X)):
        ms = ctx.cg_update_time(arith, nrep=20)
        gbs = 288.0 * Vh / (ms * 1e-3) * 1e-9
        upd[label] = {"ms": ms, "gbs": gbs, "frac_of_hbm": gbs / hbm}
    res["cg_update_48x4"] = {"bytes_per_site": 288, "kernels": upd, "paper_a100_gbs": PAPER_TABLE1_A100_GBS,
                             "paper_a100_frac": PAPER_TABLE1_A100_GBS / 1555.0}
    ctx.close()
    return res


def section_force(stag, torch, timer, hbm):
    """64^3 x 16, eps = 0.3, m = 0.01: force kernel given X, and the autograd forward + backward."""
    w = li.WORKLOADS[5]
    dims, mass = w["dims"], w["mass"]
    ctx = stag.Context(dims)
    U = li.random_links_torch(dims, "smooth", w["eps"], seed=li.workload_seed(5, 0))
    ctx.upload_gauge(U)
    phi = li.gaussian_half_torch(dims, seed=li.workload_seed(5, 1))
    S, X, st = ctx.fermion_action(phi, mass, tol=TOL, inner_prec=0)
    P = torch.empty_like(U)
    ms_f, _ = timer(lambda: ctx.fermion_force(X, P=P), reps=5, warm=2)
    nlinks = 4 * ctx.V
    # per link: the link read (144 B) and P written (144 B); X and Y read once per site (96 B per 4 links)
    bpl = 144 + 144 + 24
    gbs = bpl * nlinks / (ms_f * 1e-3) * 1e-9
    res = {"workload": w["name"] + " (inputs from the torch generator)",
           "force_call_ms": ms_f, "links": nlinks, "algorithmic_bytes_per_link": bpl, "achieved_gbs": gbs,
           "frac_of_hbm": gbs / hbm, "action_solve_iters": st["iters"],
           "force_note": "stag_fermion_force with P only: the exponent of X and its double-float split, "
                         "Y' = D_oe X' by the double-float operator, and the force kernel on those fields "
                         "(P in double-float arithmetic, accumulated in double)"}
    Ug = U.clone().requires_grad_(True)

    def fwd_bwd():
        S = stag.StaggeredAction(Ug, phi, ctx, mass, tol=TOL)   # default solver: mixed, float 18-real inner
        S.backward()
        return S

    ms_ab, _ = timer(fwd_bwd, reps=1)
    res["autograd_forward_backward_ms"] = ms_ab
    res["autograd_note"] = "forward solves X; backward re-solves X (not stored) and applies the force kernel"

    def fwd_bwd_half():
        # the same with the solver options SU(3) links allow: half 12-real inner
        # iteration in temporal gauge (double-float reliable updates, 1e-10)
        S = stag.StaggeredAction(Ug, phi, ctx, mass, tol=TOL, inner_prec=stag.F16, inner_recon=12,
                                 temporal_gauge=1)
        S.backward()
        return S

    ms_ah, _ = timer(fwd_bwd_half, reps=1)
    res["autograd_forward_backward_half12_temporal_gauge_ms"] = ms_ah
    ctx.close()
    del Ug, U, P
    torch.cuda.empty_cache()
    return res


# ---------------------------------------------------------------- ours

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="headline step only (no workload sections)")
    ap.add_argument("--use-graph", type=int, default=1,
                    help="1: device-side loop in one CUDA graph; 0: host-driven loop (per-kernel profiling)")
    ap.add_argument("--f64-arith", type=int, default=F64_IEEE, choices=[F64_IEEE, F64X],
                    help="arithmetic of the headline solve (0 IEEE double, the default; 3 double-float)")
    ap.add_argument("--sweep-multi", default=None, metavar="LXxLYxLZxLT",
                    help="time every multi-vector configuration (the link-tile split G x NBT and the "
                         "register-blocked blocks) for n = 1, 2, 4, 8, 16 vectors, float and half 12-real, one "
                         "JSON line per (storage, n); CUDA events, L2 flushed before each launch")
    ap.add_argument("--profile-kernel", default=None,
                    help="only run a few launches of one operator on the workload (for ncu): "
                         "dslash_f64_18, dslash_f64x_18, dslash_f32_12, dslash_f16_12, ..., dslash_all (one launch "
                         "of each storage), or whole host-driven solves cg_f64 / cg_f64x, multi_f32_12 / "
                         "multishift_f32_12 (32^3 x 16), mixed_f16_12 / mixed_f32_12 (48^3 x 12), or force "
                         "(32^3 x 16); a _tg suffix on an operator or mixed mode selects the temporal-gauge "
                         "links; optional @LXxLYxLZxLT")
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
    if args.sweep_multi:
        return sweep_multi(args, stag, torch)

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
    flush = L2Flush(torch, dev)
    stream = torch.cuda.current_stream()
    timer = Timer(torch, flush)
    peaks, peak_kind = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    ug, arith = args.use_graph, args.f64_arith

    def barrier():
        if ws > 1:
            dist.barrier()

    for _ in range(args.warmup):
        st = ctx.cg_solve(x, b, mass, tol=TOL, use_graph=ug, f64_arith=arith)
    torch.cuda.synchronize()

    # ---- timed region: K complete solves, L2 flushed between them
    times, stats = [], []
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = ctx.cg_solve(x, b, mass, tol=TOL, use_graph=ug, f64_arith=arith)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            stats.append(st)
    torch.cuda.synchronize()
    barrier()
    t_sum = max_over_ranks(sum(times), ws, dev)
    ms_per_step = t_sum / args.steps
    half_per_step = statistics.mean(half_dslash(s) for s in stats)
    value = weak_scaling_value(ws, Vh, half_per_step, ms_per_step)
    df_dir = cg_df_dir(Vh, getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 126 << 20))
    launches = sum(cg_kernel_launches(s, ug, arith, df_dir) for s in stats)
    clocks = clk.summary()
    x_ieee = x.clone()

    # ---- the other arithmetics on the same system: double-float, temporal
    # gauge (6 link reads per site, the paper's storage), mixed precision
    arms = {}
    ms_df, st_df = timer(lambda: ctx.cg_solve(x, b, mass, tol=TOL, use_graph=ug, f64_arith=F64X), reps=3)
    arms["cg_f64x"] = {"arithmetic": "double storage, double-float (f32x2) operator and BLAS, double reductions",
                       "time_to_solution_ms": ms_df, "iters": st_df["iters"],
                       "true_rel_residual": st_df["true_rel_residual"], "speedup_vs_ieee_f64": ms_per_step / ms_df,
                       "rel_diff_to_ieee_solution": float(torch.linalg.norm(x - x_ieee) / torch.linalg.norm(x_ieee))}
    tg_note = ("; links in temporal gauge (Sec. 4.3): U' = g U g^dagger with the time links 1 off the last "
               "slice, 6 + 2/Lt link reads per site, solving M' x' = g b and returning g^dagger x'")
    for name, a in (("cg_f64x_temporal_gauge", F64X), ("cg_f64_temporal_gauge", F64_IEEE)):
        ctx.cg_solve(x, b, mass, tol=TOL, use_graph=ug, f64_arith=a, temporal_gauge=1)   # builds the transform once
        ms_tg, st_tg = timer(lambda: ctx.cg_solve(x, b, mass, tol=TOL, use_graph=ug, f64_arith=a,
                                                  temporal_gauge=1), reps=3)
        arms[name] = {
            "arithmetic": ("as cg_f64x" if a == F64X else "IEEE double as the headline") + tg_note,
            "time_to_solution_ms": ms_tg, "iters": st_tg["iters"], "true_rel_residual": st_tg["true_rel_residual"],
            "speedup_vs_ieee_f64": ms_per_step / ms_tg}
    for name, prec, tg in (("mixed_f32_12", stag.F32, 0), ("mixed_f16_12", stag.F16, 0),
                           ("mixed_f32_12_temporal_gauge", stag.F32, 1), ("mixed_f16_12_temporal_gauge", stag.F16, 1)):
        m, sm = timer(lambda: ctx.cg_solve_mixed(x, b, mass, tol=TOL, inner_prec=prec, inner_recon=12,
                                                 use_graph=ug, temporal_gauge=tg), reps=3)
        arms[name] = {"arithmetic": f"{'float' if prec == stag.F32 else 'half + per-site norm'} 12-real inner "
                                    "iteration, double-float reliable updates, double solution" + (tg_note if tg else ""),
                      "time_to_solution_ms": m, "iters": sm["iters"], "reliable_updates": sm["reliable_updates"],
                      "true_rel_residual": sm["true_rel_residual"], "speedup_vs_ieee_f64": ms_per_step / m}

    # ---- the dominant kernel, standalone: per-launch CUDA events, L2 flushed before each
    psi = torch.from_numpy(li.gaussian_half(dims, seed=99)).to(dev)
    out = ctx.new_half()
    kern = {"f64_18": dslash_kernel_entry(timer, ctx, psi, out, F64_IEEE, 18, Vh, hbm),
            "f64x_18": dslash_kernel_entry(timer, ctx, psi, out, F64X, 18, Vh, hbm),
            "f32_12": dslash_kernel_entry(timer, ctx, psi, out, stag.F32, 12, Vh, hbm),
            "f16_12": dslash_kernel_entry(timer, ctx, psi, out, stag.F16, 12, Vh, hbm),
            "f64_18_temporal_gauge": dslash_kernel_entry(timer, ctx, psi, out, F64_IEEE, 18, Vh, hbm, tg=True),
            "f64x_18_temporal_gauge": dslash_kernel_entry(timer, ctx, psi, out, F64X, 18, Vh, hbm, tg=True),
            "f32_12_temporal_gauge": dslash_kernel_entry(timer, ctx, psi, out, stag.F32, 12, Vh, hbm, tg=True),
            "f16_12_temporal_gauge": dslash_kernel_entry(timer, ctx, psi, out, stag.F16, 12, Vh, hbm, tg=True)}
    traffic = load_traffic()
    fp64_probe = stag.fma_probe(stag.F64) * 1e3
    fp32_probe = stag.fma_probe(stag.F32) * 1e3
    if arith == F64_IEEE:
        mk = kern["f64_18"]
        peak = fp64_peak_gflops()
        roofline = {"kernel": "k_dslash<LinkField<double2,18>, SpinorF64, SpinorF64> (the IEEE-double operator of "
                              "the CG; stag_dslash_repeat, STAG_F64)",
                    "bound": "alu", "achieved": mk["gflops"], "peak": peak, "unit": "GFLOP/s",
                    "frac": mk["gflops"] / peak, "traffic": traffic.get("dslash_f64_18_48c12"),
                    "peak_source": "FP64 FMA rate from unit counts and max clock: 152 SM x 2 DFMA/clk x 2 flop x "
                                   "2.07 GHz",
                    "peak_probe_gflops": fp64_probe,
                    "frac_of_probe": mk["gflops"] / fp64_probe,
                    "hbm": {"achieved_gbs": mk["achieved_gbs"], "peak_gbs": hbm, "frac": mk["achieved_gbs"] / hbm,
                            "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind} copy bandwidth)"},
                    "algorithmic_flop_per_launch": FLOP_PER_SITE * Vh,
                    "algorithmic_bytes_per_launch": mk["algorithmic_bytes_per_site"] * Vh,
                    "kernel_ms": mk["ms"]}
    else:
        mk = kern["f64x_18"]
        roofline = {"kernel": "k_dslash<LinkFieldDF<18>, SpinorDF, SpinorDF> (the double-float operator on its "
                              "double-float vectors; stag_dslash_repeat, STAG_F64X)",
                    "bound": "hbm", "achieved": mk["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                    "frac": mk["achieved_gbs"] / hbm, "traffic": traffic.get("dslash_f64x_df_18_48c12"),
                    "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind} copy bandwidth)",
                    "algorithmic_bytes_per_launch": mk["algorithmic_bytes_per_site"] * Vh, "kernel_ms": mk["ms"]}

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region
    b_host = torch.from_numpy(b_np).pin_memory()
    x_host = torch.empty_like(b_host).pin_memory()
    xd = ctx.new_half()
    bd = torch.empty_like(xd)
    e2e_t, e2e_half = [], []
    for _ in range(max(3, args.steps // 4)):
        flush(3.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bd.copy_(b_host, non_blocking=True)
        st = ctx.cg_solve(xd, bd, mass, tol=TOL, use_graph=ug, f64_arith=arith)
        x_host.copy_(xd, non_blocking=True)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
        e2e_half.append(half_dslash(st))
    e2e_val = FLOP_PER_SITE * Vh * statistics.mean(e2e_half) / statistics.mean(e2e_t) * 1e-9

    sections = {}
    if rank == 0 and ws == 1 and not args.quick:
        ctx.close()
        for name, fn in (("w32c8", lambda: section_32c8(stag, torch, timer, hbm)),
                         ("w32c16", lambda: section_32c16(stag, torch, timer)),
                         ("force_64c16", lambda: section_force(stag, torch, timer, hbm)),
                         ("paper_tables", lambda: section_paper_tables(stag, torch, timer, hbm))):
            try:
                sections[name] = fn()
            except Exception as e:   # a failed section is reported, not hidden
                sections[name] = {"error": repr(e)}

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
        "dtype": "f64" if arith == F64_IEEE else "f64 storage; operator in double-float (f32x2)",
        "data": "synthetic",
        "config": headline_config(w),
        "cg": {"time_to_solution_ms": ms_per_step, "iters": last["iters"], "restarts": last["restarts"],
               "true_rel_residual": last["true_rel_residual"], "half_dslash_per_solve": half_per_step,
               "f64_arith": "IEEE double (STAG_F64)" if arith == F64_IEEE else "double-float (STAG_F64X)"},
        "arms_48c12": arms,
        "roofline": roofline,
        "dslash_kernels_48c12": kern,
        "alu_probes": {"fp64_fma_gflops": fp64_probe, "fp32_fma_gflops": fp32_probe,
                       "note": "stag_fma_probe: independent FMA chains on every SM, CUDA events"},
        "e2e": {"value": e2e_val, "unit": "GFLOP/s", "h2d_bytes_per_step": int(b_host.numel() * 16),
                "d2h_bytes_per_step": int(x_host.numel() * 16), "seconds_per_step": statistics.mean(e2e_t)},
        "sections": sections,
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
