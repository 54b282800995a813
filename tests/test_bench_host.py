"""Host-side pieces of bench.py: the paper's counts (Sec. 4.3) that the
measurement accounting relies on, and the multi-rank aggregation, run as two
gloo ranks on the CPU."""

import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def read_golden():
    vals = {}
    with open(os.path.join(ROOT, "tests", "golden", "paper_counts.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


def test_flop_and_float_counts_match_the_paper():
    import bench
    g = read_golden()
    # 570 flop per site: per direction two complex 3x3 mat-vecs (9 complex
    # multiplies of 6 flop + 6 complex adds of 2 flop) and one 3-vector add,
    # plus the 3 adds of the four direction sums
    matvec = 9 * 6 + 6 * 2
    assert 4 * (2 * matvec + 3 * 2) + 3 * 3 * 2 == g["flop_per_site"] == bench.FLOP_PER_SITE
    assert bench.paper_float_count(1) == g["floats_per_site"]
    assert abs(bench.paper_arithmetic_intensity(1, 8) - g["ai_fp64"]) < 0.005
    assert abs(bench.paper_arithmetic_intensity(1, 4) - g["ai_fp32"]) < 0.005


def test_compulsory_bytes():
    import bench
    assert bench.dslash_bytes_per_site(8, 18) == 1248
    assert bench.dslash_bytes_per_site(8, 12) == 864
    assert bench.dslash_bytes_per_site(4, 12) == 432
    # temporal gauge (Sec. 4.3): 6 + 2/Lt links per site, spinors as before
    assert bench.dslash_bytes_per_site_tg(8, 18, 12) == 984
    assert bench.dslash_bytes_per_site_tg(4, 12, 12) == 344
    assert bench.dslash_bytes_per_site_tg(2, 12, 12) + 8 == 180
    # at Lt = 2 every site sits next to the boundary: 7 links per site on average
    assert bench.dslash_bytes_per_site_tg(4, 12, 2) == 7 * 48 + 48


def test_weak_scaling_value():
    import bench
    v1 = bench.weak_scaling_value(1, 131072, 162, 13.0)
    assert abs(v1 - 570 * 131072 * 162 / 13e-3 * 1e-9) < 1e-6
    assert abs(bench.weak_scaling_value(4, 131072, 162, 13.0) - 4 * v1) < 1e-6


def _rank(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import sys
    sys.path.insert(0, ROOT)
    import bench
    q.put((rank, bench.max_over_ranks(10.0 + 5 * rank, ws)))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get() for _ in range(2))
    assert got == {0: 15.0, 1: 15.0}


def test_cg_kernel_launch_count():
    import bench
    # normalisation of b (3) + start (1) + iterations + residual pair per pass
    # + restart kernels + scaled copy of the solution (1)
    # graph: iterations run in whole bodies of CG_GRAPH_UNROLL
    st = {"iters": 80, "restarts": 0}
    assert bench.cg_kernel_launches(st, 1) == 4 + 4 * 80 + 2 + 1
    st = {"iters": 81, "restarts": 0}
    assert bench.cg_kernel_launches(st, 1) == 4 + 4 * 84 + 2 + 1
    # host loop: whole batches of CG_CHECK_EVERY
    assert bench.cg_kernel_launches({"iters": 80, "restarts": 0}, 0) == 4 + 4 * 100 + 2 + 1
    # a restart adds a pass: its residual kernels and the restart kernel
    assert bench.cg_kernel_launches({"iters": 2, "restarts": 1}, 1) == 4 + 4 * 8 + 4 + 1 + 1

    # the double-float solver: three kernels per iteration (four with the
    # direction update as a pass of its own)
    assert bench.cg_kernel_launches({"iters": 80, "restarts": 0}, 1, 3) == 4 + 3 * 80 + 2 + 1
    assert bench.cg_kernel_launches({"iters": 80, "restarts": 0}, 1, 3, False) == 4 + 4 * 80 + 2 + 1


def test_cg_direction_update_rule(monkeypatch):
    import bench
    l2 = 126 << 20
    monkeypatch.delenv("STAG_CG_DIR", raising=False)
    assert bench.cg_df_dir(32 * 32 * 32 * 8 // 2, l2)          # 31.5 MB of vectors
    assert not bench.cg_df_dir(48 * 48 * 48 * 12 // 2, l2)     # 159 MB
    monkeypatch.setenv("STAG_CG_DIR", "0")
    assert not bench.cg_df_dir(128, l2)
    monkeypatch.setenv("STAG_CG_DIR", "1")
    assert bench.cg_df_dir(48 * 48 * 48 * 12 // 2, l2)


def test_clock_sampler_keeps_samples_of_the_timed_window(tmp_path, monkeypatch):
    """The sampler waits for its first sample before the timed region and keeps
    only the samples taken inside it (a fake nvidia-smi on PATH, no GPU)."""
    import time
    import bench
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/usr/bin/env python3\n"
                    "import sys, time\n"
                    "time.sleep(0.3)\n"
                    "k = 0\n"
                    "while True:\n"
                    "    act = 'Active' if k == 3 else 'Not Active'\n"
                    "    print(f'0, {1900 + k}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, {act}', flush=True)\n"
                    "    k += 1\n"
                    "    time.sleep(0.05)\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}:{os.environ['PATH']}")
    with bench.ClockSampler(0) as clk:
        assert clk.samples, "entering waits for the first sample"
        time.sleep(0.4)
    s = clk.summary()
    assert s["samples"] >= 4
    assert s["sm_max_mhz"] == 2070.0 and 1900.0 <= s["sm_mhz"] <= 1930.0
    assert s["reasons"] == ["sw_power_cap"]


def test_reference_arm_line(tmp_path):
    """`bench.py --impl reference` times the CPU oracle on the benchmark's
    workload and prints one JSON line with the keys the harness reads, the
    same metric, unit and config as the GPU arm."""
    import json
    import subprocess
    import sys
    import bench
    import lattice_inputs as li
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=str(tmp_path))
    assert p.returncode == 0, p.stderr
    line = json.loads(p.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "GFLOP/s"
    assert line["higher_is_better"] is True and line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 3
    assert line["config"] == bench.headline_config(li.WORKLOADS[bench.WORKLOAD_INDEX])
    cb = line["cpu_baseline"]
    import oracle
    with oracle.threads():
        cores = oracle.num_threads()
    assert cb["kind"] == "oracle" and cb["cores"] == cores and cb["value"] == line["value"] and cb["sample"]
    assert line["dtype"] == "f64" and line["config"]["dims"] == [48, 48, 48, 12]
    assert line["e2e"] == {"value": line["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
