"""Benchmark of the PW advection tendency path on GB300.

One step = one pass of the hot path: the source terms su, sv, sw of the PW
scheme over one 2048 x 2048 x 64 FP32 grid (268M interior cells; 512 x 512 x 64
with --workload 512), inputs resident in HBM, one TMA k-march kernel launch.
Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload 2048|512]

N > 1 (torchrun): every rank runs its own independent grid of the same size
(independent problems, no data-path collective; weak scaling); the timed
region is bracketed by a barrier and the max over ranks is reported.

--impl reference times the CPU oracle (plain C loop nest, FP64, one thread)
on bounded slabs of the same workload, on rank 0 only.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "PW advection Gcell/s & % of HBM peak; FP32 vs BF16-stored at stated error"
BYTES_PER_CELL_F32 = 24          # read u, v, w + write su, sv, sw (4 bytes each)
FLOPS_PER_CELL = 63              # 21 useful FLOPs per field (Sec. 4 op structure)
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "pw_tend_tma_f32_2048x2048x64.md")
KERNEL_SOURCE = os.path.join(ROOT, "paper_2301_13016_gb300", "csrc", "pw_tend.cu")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["2048", "512"], default="2048")
    p.add_argument("--e2e-steps", type=int, default=5)
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


def workload(name):
    n = int(name)
    return dict(nx=n, ny=n, nz=64)


def workload_label(w):
    return (f"PW tendencies FP32, {w['nx']}x{w['ny']}x{w['nz']} interior + 1 halo, periodic x/y, rigid lid; "
            "u,v,w = 10*N(0,1) m/s seeded (2301-2303); dx=dy=100 m; dz 20->200 m")


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if (args.impl == "ours" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available() and args.impl == "ours":
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    with open(KERNEL_SOURCE, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the TMA kernel from the committed ncu summary,
    if it was taken on the current kernel source (else None)."""
    try:
        text = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    m_hash = re.search(r"kernel source sha256\[:16\]:\s*`?([0-9a-f]{16})", text)
    m_bytes = re.search(r"dram bytes per launch \(read\+write\):\s*([0-9.eE+]+)", text)
    if not m_hash or not m_bytes or m_hash.group(1) != kernel_source_hash():
        return None
    return float(m_bytes.group(1))


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        self.t0 = time.time()

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.strip()]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() in ("active", "1"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(w, budget_s=10.0):
    """The CPU oracle (FP64 plain C loop nest, one thread) on slabs of the
    same workload: nx x 128 x nz grids from the same generator, repeated
    until about budget_s seconds of CPU work."""
    import oracle
    from paper_2301_13016_gb300 import inputs
    nx, nz = w["nx"], w["nz"]
    ny = 128
    c = inputs.make_coeffs(nz)
    f = [x.numpy().astype(np.float64) for x in inputs.random_fields(nx, ny, nz)]
    oracle.tendencies(*f, c)                      # load + warm
    cells, t_used, reps = 0, 0.0, 0
    while t_used < budget_s and reps < 200:
        t = time.perf_counter()
        oracle.tendencies(*f, c)
        t_used += time.perf_counter() - t
        cells += nx * ny * nz
        reps += 1
    return {"value": cells / t_used / 1e9, "unit": "Gcell/s", "cores": 1, "kind": "oracle",
            "sample": f"FP64 oracle on {reps} x ({nx}x{ny}x{nz}) slabs of the same workload, "
                      f"{t_used:.1f} s CPU, single thread"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = workload(args.workload)
    import oracle
    from paper_2301_13016_gb300 import inputs
    nx, nz = w["nx"], w["nz"]
    ny = 64
    c = inputs.make_coeffs(nz)
    f = [x.numpy().astype(np.float64) for x in inputs.random_fields(nx, ny, nz)]
    for _ in range(max(args.warmup, 0)):
        oracle.tendencies(*f, c)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.tendencies(*f, c)
    dt = time.perf_counter() - t
    cells = nx * ny * nz * args.steps
    val = cells / dt / 1e9
    sample = f"FP64 oracle, one thread, per step one {nx}x{ny}x{nz} slab of the {w['nx']}x{w['ny']}x{w['nz']} workload"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Gcell/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_label(w), "nx": w["nx"], "ny": w["ny"],
                                            "nz": w["nz"], "sample_ny": ny},
            "cpu_baseline": {"value": val, "unit": "Gcell/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "Gcell/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local):
    import paper_2301_13016_gb300 as pwlib
    from paper_2301_13016_gb300 import inputs
    w = workload(args.workload)
    nx, ny, nz = w["nx"], w["ny"], w["nz"]
    c = inputs.make_coeffs(nz)
    grid = pwlib.Grid(nx, ny, nz)
    h = pwlib.PW(grid, c)
    # inputs generated on the device by torch's generator (seeded per rank)
    dense = inputs.random_fields(nx, ny, nz, device="cuda",
                                 seeds=tuple(s + 1000 * rank for s in (2301, 2302, 2303)))
    dev = [grid.from_dense(x) for x in dense]
    del dense
    outs = [grid.alloc(fill=0.0) for _ in range(3)]
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        h.tendencies(*dev, *outs, stream=stream)
    h.sync(stream)
    assert h.last_kernel == 2, "the benchmark must run the TMA k-march kernel"

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        h.tendencies(*dev, *outs, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    h.sync(stream)
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(ms, world)
    cells = grid.cells
    value = cells * args.steps * world / (ms / 1e3) / 1e9            # Gcell/s, whole job
    launch_s = ms / 1e3 / args.steps                                  # one kernel per step
    algo_bytes = BYTES_PER_CELL_F32 * cells
    peak, peak_kind = measured_peak()
    achieved = algo_bytes / launch_s / 1e9

    # end to end through the host-buffer entry point: H2D + kernel + D2H per step
    hin = [t.cpu().pin_memory() for t in dev]
    hout = [torch.zeros(grid.alloc_elems, dtype=torch.float32).pin_memory() for _ in range(3)]
    del dev, outs
    torch.cuda.empty_cache()
    h.tendencies_host(*hin, *hout, stream=stream)          # warm (allocates staging)
    barrier(world)
    t = time.perf_counter()
    for _ in range(args.e2e_steps):
        h.tendencies_host(*hin, *hout, stream=stream)
    e2e_s = max_over_ranks(time.perf_counter() - t, world)
    span = (grid.origin + nz * grid.pitch_k + (ny + 1) * grid.pitch_j + nx + 2) - \
        (grid.origin + grid.pitch_k + 0 * grid.pitch_j + 0)
    span_bytes = span * 4
    e2e = {"value": cells * args.e2e_steps * world / e2e_s / 1e9, "unit": "Gcell/s",
           "h2d_bytes_per_step": 3 * span_bytes, "d2h_bytes_per_step": 3 * span_bytes,
           "steps": args.e2e_steps}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "Gcell/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_label(w), "nx": nx, "ny": ny, "nz": nz, "cells_per_gpu": cells,
                   "l2": "inputs larger than L2 (3 x %.2f GB resident per grid)" % (grid.alloc_elems * 4 / 1e9),
                   "kernel": "TMA k-march (pw_tendencies, automatic launch shape)",
                   "parallelism": f"{world} independent grids, one per GPU"},
        "hbm_frac_of_measured": achieved / peak,
        "gflops_useful": value * FLOPS_PER_CELL,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": profiled_traffic(),
                     "peak_kind": peak_kind, "algorithmic_bytes_per_launch": algo_bytes},
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_init(args)
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
