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

--impl reference times the CPU oracle (plain C loop nest, FP64, unchanged)
on bounded slabs of the same workload, one thread per host core, on rank 0
only.  --form selects another form of the path (16-bit storage, fused steps,
two steps per pass, batch, adjoint rollout, small-grid latency, host link).
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
NOMINAL_HBM_GBS = 8000.0         # GB300 HBM3e, nominal (about 8 TB/s)
BYTES_PER_CELL_F32 = 24          # read u, v, w + write su, sv, sw (4 bytes each)
FLOPS_PER_CELL = 63              # 21 useful FLOPs per field (Sec. 4 op structure)
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "pw_tend_tma_f32_2048x2048x64.md")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2301_13016_gb300", "csrc", f)
                  for f in ("pw_stencil.cuh", "pw_device.cuh", "pw_tend.cu")]
FORMS = ["tend", "tend-bf16", "tend-f16", "step", "step-bf16", "step2", "step2-bf16", "step2-f16",
         "batch", "batch-bf16", "adjoint", "latency64", "hostlink", "step-slab"]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["2048", "512"], default="2048")
    p.add_argument("--e2e-steps", type=int, default=5)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--batch-grids", type=int, default=512, help="batch form: number of grids")
    p.add_argument("--batch-tile", default="", help="batch form: LANES,TY,STAGES,CTAS_PER_SM[,ROWS[,CELLS]] (skips the autotuner)")
    p.add_argument("--skip-fp32-ref", action="store_true",
                   help="forms: do not time the FP32 tendency form beside them (small profiling runs)")
    p.add_argument("--form", choices=FORMS, default="tend",
                   help="tend (default: the headline FP32 tendency benchmark) or another form of the path")
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


def whole_job_rate(units_per_rank, world, seconds_max):
    """Weak scaling: every rank processes units_per_rank in its own time; the
    job rate is all ranks' units over the slowest rank's time (units/s)."""
    return units_per_rank * world / seconds_max


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
    """sha256[:16] of the tendency kernel's sources with comments and
    whitespace removed, so that only a change to the code voids a profile."""
    h = hashlib.sha256()
    for path in KERNEL_SOURCES:
        with open(path) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update("".join(text.split()).encode())
    return h.hexdigest()[:16]


def source_version():
    """Which code produced this line: the git commit when the checkout has its
    .git directory (read from the files, no git process), and always the
    sha256[:16] of the product sources (package, header, oracle, this file),
    which a checkout of any commit reproduces with the same function."""
    git_sha = None
    try:
        head = open(os.path.join(ROOT, ".git", "HEAD")).read().strip()
        if head.startswith("ref: "):
            ref = head[5:]
            path = os.path.join(ROOT, ".git", ref)
            if os.path.exists(path):
                git_sha = open(path).read().strip()
            else:
                for ln in open(os.path.join(ROOT, ".git", "packed-refs")):
                    if ln.strip().endswith(" " + ref):
                        git_sha = ln.split()[0]
        else:
            git_sha = head
    except OSError:
        pass
    files = []
    for sub, exts in (("paper_2301_13016_gb300", (".py", ".cu", ".cuh", ".h")), ("include", (".h",)),
                      ("oracle", (".c", ".h", ".py"))):
        for dirpath, dirnames, names in os.walk(os.path.join(ROOT, sub)):
            dirnames[:] = sorted(d for d in dirnames if not d.startswith(("_", ".")))
            files += [os.path.join(dirpath, n) for n in names if n.endswith(exts)]
    files += [os.path.join(ROOT, "bench.py"), os.path.join(ROOT, "__graft_entry__.py")]
    h = hashlib.sha256()
    for path in sorted(files):
        h.update(os.path.relpath(path, ROOT).encode() + b"\0")
        with open(path, "rb") as fh:
            h.update(fh.read())
    return {"git_sha": git_sha, "source_sha256": h.hexdigest()[:16]}


def host_numa():
    """NUMA nodes of the host and the node nvidia-smi and sysfs give for GPU 0
    (where pinned host buffers should sit for the host link)."""
    out = {"nodes": None, "gpu_node": None}
    try:
        out["nodes"] = len([d for d in os.listdir("/sys/devices/system/node") if re.fullmatch(r"node\d+", d)])
        bus = subprocess.run(["nvidia-smi", "--query-gpu=pci.bus_id", "--format=csv,noheader", "-i", "0"],
                             capture_output=True, text=True, timeout=30).stdout.strip().lower()
        dom, rest = bus.split(":", 1)
        path = f"/sys/bus/pci/devices/{int(dom, 16):04x}:{rest}/numa_node"
        with open(path) as fh:
            out["gpu_node"] = int(fh.read().strip())
    except Exception:
        pass
    return out


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


def cpu_baseline(w, budget_s=10.0, slab=None):
    """The CPU oracle (plain C loop nest, unchanged) on slabs of the same
    workload: nx x 128 x nz grids, repeated until about budget_s seconds of
    CPU work in all: FP64 on every host core at once (the value), and beside
    it FP32 on every core and FP64 / FP32 on one thread.  With `slab` (rows 1..128 of the benchmark's own inputs, with
    their halo rows, and the GPU's FP32 and BF16-storage source terms on those
    rows) the slab is the sample, and its first oracle result is also the
    reference the GPU outputs are checked against: max|err| / max|ref| per
    field, the largest of the three reported."""
    import oracle
    from paper_2301_13016_gb300 import inputs
    nx, nz = w["nx"], w["nz"]
    ny = 128
    c = inputs.make_coeffs(nz)
    parity = None
    if slab is None:
        f = [x.numpy().astype(np.float64) for x in inputs.random_fields(nx, ny, nz)]
        oracle.tendencies(*f, c)                      # load + warm
    else:
        f = slab["inputs"]
        ref = oracle.tendencies(*f, c)
        parity = {"sample": f"rows 1..{ny} of the workload (all {nx} columns, {nz} levels), FP64 oracle"}
        for key, got in slab["outputs"].items():
            parity[key] = max(float(np.abs(g - r[1:-1, 1:-1, 1:-1]).max() / np.abs(r[1:-1, 1:-1, 1:-1]).max())
                              for g, r in zip(got, ref))
    slab_cells = nx * ny * nz

    def single(precision, budget):
        args = f if precision == "f64" else [x.astype(np.float32) for x in f]
        cells, t_used, reps = 0, 0.0, 0
        while t_used < budget and reps < 200:
            t = time.perf_counter()
            oracle.tendencies(*args, c, precision=precision)
            t_used += time.perf_counter() - t
            cells += slab_cells
            reps += 1
        return cells / t_used / 1e9, reps, t_used

    def all_cores(budget, precision="f64"):
        # the same single-thread oracle on every host core at once: its C
        # loop runs outside the interpreter lock, one call per thread
        import concurrent.futures as cf
        n = len(os.sched_getaffinity(0))
        args = f if precision == "f64" else [x.astype(np.float32) for x in f]
        deadline = time.perf_counter() + budget

        def worker(_):
            done = 0
            while time.perf_counter() < deadline:
                oracle.tendencies(*args, c, precision=precision)
                done += 1
            return done
        t = time.perf_counter()
        with cf.ThreadPoolExecutor(max_workers=n) as ex:
            calls = sum(ex.map(worker, range(n)))
        return calls * slab_cells / (time.perf_counter() - t) / 1e9, n, calls

    v64, reps, t_used = single("f64", budget_s * 0.4)
    v32, reps32, t32 = single("f32", budget_s * 0.15)
    vall, n, calls = all_cores(budget_s * 0.3)
    vall32, _, calls32 = all_cores(budget_s * 0.15, "f32")
    out = {"value": vall, "unit": "Gcell/s", "cores": n, "kind": "oracle",
           "sample": f"FP64 oracle on ({nx}x{ny}x{nz}) slabs of the same workload: {calls} calls spread over "
                     f"{n} threads (one per host core) for {budget_s * 0.3:.1f} s",
           "all_cores_f32": vall32, "all_cores_f32_calls": calls32,
           "single_thread_f64": v64, "single_thread_f32": v32,
           "single_thread_sample": f"{reps} FP64 calls in {t_used:.1f} s, {reps32} FP32 calls in {t32:.1f} s"}
    if parity is not None:
        out["parity"] = parity
    return out


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle (FP64 plain C loop nest, untuned) on
    the host cores, one 2048 x 64 x 64 slab of the workload per core per step,
    the cores working at once (threads: the oracle's C loop runs outside the
    interpreter lock)."""
    if rank != 0:
        return
    import concurrent.futures as cf
    w = workload(args.workload)
    import oracle
    from paper_2301_13016_gb300 import inputs
    nx, nz = w["nx"], w["nz"]
    ny = 64
    c = inputs.make_coeffs(nz)
    f = [x.numpy().astype(np.float64) for x in inputs.random_fields(nx, ny, nz)]
    n = len(os.sched_getaffinity(0))
    with cf.ThreadPoolExecutor(max_workers=n) as ex:
        step = lambda: list(ex.map(lambda _: oracle.tendencies(*f, c), range(n)))
        for _ in range(max(args.warmup, 0)):
            step()
        t = time.perf_counter()
        for _ in range(args.steps):
            step()
        dt = time.perf_counter() - t
    cells = nx * ny * nz * n * args.steps
    val = cells / dt / 1e9
    sample = (f"FP64 oracle, {n} threads (one per host core), per step one {nx}x{ny}x{nz} slab of the "
              f"{w['nx']}x{w['ny']}x{w['nz']} workload per thread")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Gcell/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_label(w), "nx": w["nx"], "ny": w["ny"],
                                            "nz": w["nz"], "sample_ny": ny},
            "cpu_baseline": {"value": val, "unit": "Gcell/s", "cores": n, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "Gcell/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "version": source_version()}
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
    for _ in range(2):   # the GPU busy again after the pause, untimed
        h.tendencies(*dev, *outs, stream=stream)
    torch.cuda.synchronize()
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
    # per-launch times (events between launches, outside the timed region above)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(min(args.steps, 50) + 1)]
    evs[0].record(stream)
    for e in evs[1:]:
        h.tendencies(*dev, *outs, stream=stream)
        e.record(stream)
    torch.cuda.synchronize()
    per = [a.elapsed_time(b) for a, b in zip(evs[:-1], evs[1:])]
    timing = {"launches": len(per), "mean_ms": statistics.mean(per), "median_ms": statistics.median(per),
              "min_ms": min(per), "max_ms": max(per)}
    cells = grid.cells
    value = whole_job_rate(cells * args.steps, world, ms / 1e3) / 1e9   # Gcell/s, whole job
    launch_s = ms / 1e3 / args.steps                                  # one kernel per step
    algo_bytes = BYTES_PER_CELL_F32 * cells
    peak, peak_kind = measured_peak()
    achieved = algo_bytes / launch_s / 1e9

    # BF16 storage of the same inputs (FP32 arithmetic), and the check slab
    bf16 = slab = None
    if rank == 0:
        rows = 128
        slab = {"inputs": [grid.view(t)[:, 0:rows + 2, :].double().cpu().numpy() for t in dev],
                "outputs": {"fp32_max_rel_err": [grid.view(o)[1:-1, 1:rows + 1, 1:-1].double().cpu().numpy()
                                                 for o in outs]}}
        g16 = pwlib.Grid(nx, ny, nz, dtype="bf16")
        h16 = pwlib.PW(g16, c)
        d16 = [g16.from_dense(grid.view(t)) for t in dev]
        o16 = [g16.alloc() for _ in range(3)]
        f16 = lambda: h16.tendencies(*d16, *o16, stream=stream)
        for _ in range(3):
            f16()
        h16.sync(stream)
        assert h16.last_kernel == 2, "the BF16 leg must run the TMA k-march kernel"
        TIMED_CLOCKS.clear()
        ms16 = _events_ms(f16, args.steps, stream)
        clocks16 = timed_clocks_summary(TIMED_CLOCKS)
        h16.sync(stream)
        slab["outputs"]["bf16_max_rel_err"] = [g16.view(o)[1:-1, 1:rows + 1, 1:-1].double().cpu().numpy()
                                               for o in o16]
        v16 = cells / (ms16 / 1e3) / 1e9
        bf16 = {"value": v16, "unit": "Gcell/s", "ms_per_step": ms16, "vs_fp32": v16 / (value / world),
                "launch_shape": h16.tma_config(), "bytes_per_cell": 12,
                "roofline_frac": 12 * cells / (ms16 / 1e3) / 1e9 / peak,
                "stated_error_bound": 1e-2, "error": "cpu_baseline.parity.bf16_max_rel_err", "clocks": clocks16}
        del h16, d16, o16
        torch.cuda.empty_cache()

    # end to end through the host-buffer entry point: H2D + kernel + D2H per step
    hin = [t.cpu().pin_memory() for t in dev]
    hout = [torch.zeros(grid.alloc_elems, dtype=torch.float32).pin_memory() for _ in range(3)]
    del dev, outs
    torch.cuda.empty_cache()
    h.tendencies_host(*hin, *hout, stream=stream)          # warm (allocates staging)
    # one call at a time (each returns with its results in host memory) ...
    barrier(world)
    t = time.perf_counter()
    for _ in range(args.e2e_steps):
        h.tendencies_host(*hin, *hout, stream=stream)
    sync_s = max_over_ranks(time.perf_counter() - t, world)
    # ... and the steps back to back through the asynchronous entry point, one
    # sync at the end: a step's inputs travel while the last step's outputs
    # come back (the reported value)
    barrier(world)
    t = time.perf_counter()
    for _ in range(args.e2e_steps):
        h.tendencies_host_async(*hin, *hout, stream=stream)
    h.sync(stream)
    e2e_s = max_over_ranks(time.perf_counter() - t, world)
    # what the host path moves: the inputs with their one-cell halo, the
    # interior of the outputs (levels 1..nz)
    e2e = {"value": whole_job_rate(cells * args.e2e_steps, world, e2e_s) / 1e9, "unit": "Gcell/s",
           "api": "pw_tendencies_host_async, steps back to back, one sync",
           "one_call_at_a_time": whole_job_rate(cells * args.e2e_steps, world, sync_s) / 1e9,
           "h2d_bytes_per_step": 3 * 4 * (nx + 2) * (ny + 2) * nz, "d2h_bytes_per_step": 3 * 4 * cells,
           "steps": args.e2e_steps, "host_numa": host_numa()}

    if rank != 0:
        return
    traffic = profiled_traffic()
    line = {
        "metric": METRIC, "value": value, "unit": "Gcell/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_label(w), "nx": nx, "ny": ny, "nz": nz, "cells_per_gpu": cells,
                   "l2": "inputs larger than L2 (3 x %.2f GB resident per grid)" % (grid.alloc_elems * 4 / 1e9),
                   "kernel": "TMA k-march (pw_tendencies, automatic launch shape)",
                   "parallelism": f"{world} independent grid{'s' if world > 1 else ''}, one per GPU"},
        "hbm_frac_of_measured": achieved / peak,
        "gflops_useful": value * FLOPS_PER_CELL,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "nominal_peak": NOMINAL_HBM_GBS,
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "traffic": traffic,
                     "traffic_bytes_per_cell": traffic / cells if traffic else None,
                     "peak_kind": peak_kind, "algorithmic_bytes_per_launch": algo_bytes,
                     "algorithmic_bytes_per_cell": BYTES_PER_CELL_F32},
        "launch_timing": timing,
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clocks,
        "bf16_storage": bf16,
        "version": source_version(),
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, slab=slab)
        if "parity" in line["cpu_baseline"]:
            line["cpu_baseline"]["parity"]["fp32_bound"] = 1e-5
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Other forms of the path (one JSON line each, rank 0, N = 1): each is timed
# beside the plain FP32 tendency kernel on the same GPU in the same process.

TIMED_CLOCKS = []   # nvidia-smi clock records of the regions _events_ms timed (this process)


def _events_ms(fn, n, stream):
    """Mean ms per call of fn over n calls, CUDA events on `stream`, with the
    SM clocks and throttle reasons sampled around the timed region."""
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    for _ in range(2):   # the GPU busy again after the pause, untimed
        fn()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        fn()
    e1.record(stream)
    e1.synchronize()
    c = sampler.stop()
    if c:
        TIMED_CLOCKS.append(c)
    return e0.elapsed_time(e1) / n


def timed_clocks_summary(records):
    """One clock record for several timed regions: the lowest median SM
    clock, the highest maximum, every throttle reason seen."""
    if not records:
        return None
    return {"sm_mhz": min(r["sm_mhz"] for r in records), "sm_max_mhz": max(r["sm_max_mhz"] for r in records),
            "reasons": sorted(set().union(*[r["reasons"] for r in records])),
            "samples": sum(r["samples"] for r in records), "regions": len(records)}


def _fp32_reference_rate(nx, ny, nz, steps, stream):
    import paper_2301_13016_gb300 as pwlib
    from paper_2301_13016_gb300 import inputs
    g = pwlib.Grid(nx, ny, nz)
    h = pwlib.PW(g, inputs.make_coeffs(nz))
    dense = inputs.random_fields(nx, ny, nz, device="cuda")
    dev = [g.from_dense(x) for x in dense]
    del dense
    outs = [g.alloc() for _ in range(3)]
    f = lambda: h.tendencies(*dev, *outs, stream=stream)
    for _ in range(5):
        f()
    ms = _events_ms(f, steps, stream)
    h.sync(stream)
    del dev, outs
    torch.cuda.empty_cache()
    return g.cells / (ms / 1e3) / 1e9


def _form_line(args, form, metric, value, unit, config, extra):
    line = {"form": form, "metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "data": "synthetic", "config": config}
    line.update(extra)
    line.setdefault("clocks", timed_clocks_summary(TIMED_CLOCKS))
    line["version"] = source_version()
    print(json.dumps(line), flush=True)


def form_tend_lowp(args, dtype):
    import paper_2301_13016_gb300 as pwlib
    from paper_2301_13016_gb300 import inputs, precision
    nx = ny = 2048
    nz = 64
    stream = torch.cuda.current_stream()
    ref = None if args.skip_fp32_ref else _fp32_reference_rate(nx, ny, nz, max(20, args.steps // 4), stream)
    c = inputs.make_coeffs(nz)
    g = pwlib.Grid(nx, ny, nz, dtype=dtype)
    h = pwlib.PW(g, c)
    dense = inputs.random_fields(nx, ny, nz, device="cuda")
    sc = precision.suggest_scales([float(x.abs().max()) for x in dense], c, dtype)
    dev = [g.from_dense(x, scale=s) for x, s in zip(dense, sc[:3])]
    del dense
    outs = [g.alloc() for _ in range(3)]
    f = lambda: h.tendencies(*dev, *outs, scale=sc, stream=stream)
    for _ in range(args.warmup):
        f()
    ms = _events_ms(f, args.steps, stream)
    h.sync(stream)
    val = g.cells / (ms / 1e3) / 1e9
    peak, kind = measured_peak()
    achieved = 12 * g.cells / (ms / 1e3) / 1e9
    _form_line(args, f"tend-{dtype}", f"PW tendencies Gcell/s, {dtype.upper()} storage (FP32 arithmetic)", val,
               "Gcell/s", {"workload": f"{nx}x{ny}x{nz} random 10*N(0,1), {dtype} storage, per-field power-of-two scales",
                           "scales": list(sc)},
               {"dtype": dtype, "ms_per_step": ms, "vs_fp32_form": val / ref if ref else None, "fp32_form_gcells": ref,
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "peak_kind": kind, "bytes_per_cell": 12},
                "gpu_launches": args.steps})


STEP2_SHAPES = [(8, 3, 1), (8, 3, 2), (8, 4, 1), (12, 3, 1), (16, 3, 1), (16, 4, 1)]


def form_step(args, dtype, spp=1):
    """Fused forward-Euler steps on 2048 x 2048 x 64 (512 x 512 x 64 with
    --workload 512, for profiling): one step per kernel pass (spp = 1, halo-1
    grid) or two (spp = 2, halo-2 grid, every instantiated launch shape timed;
    the value is the automatic shape's)."""
    import paper_2301_13016_gb300 as pwlib
    from paper_2301_13016_gb300 import inputs, precision
    nx = ny = int(args.workload)
    nz = 64
    stream = torch.cuda.current_stream()
    ref = None if args.skip_fp32_ref else _fp32_reference_rate(nx, ny, nz, max(20, args.steps // 4), stream)
    c = inputs.make_coeffs(nz)
    g = pwlib.Grid(nx, ny, nz, dtype=dtype, halo=spp)
    h = pwlib.PW(g, c)
    h.set_step_blocking(spp)
    dense = inputs.smooth_fields(nx, ny, nz, w_zero=True, device="cuda")
    sc = precision.suggest_scales([max(float(x.abs().max()), 1.0) for x in dense], c, dtype)[:3]
    q = [g.from_dense(x, scale=s) for x, s in zip(dense, sc)]
    del dense
    tmp = [g.alloc() for _ in range(3)]
    nsteps = args.steps if args.steps % (2 * spp) == 0 else args.steps + 2 * spp - args.steps % (2 * spp)
    f = lambda: h.step(*q, *tmp, 0.0, nsteps, scale=sc, stream=stream)

    def timed():
        h.step(*q, *tmp, 0.0, 2 * spp, scale=sc, stream=stream)
        ms_ = _events_ms(f, 1, stream) / nsteps
        h.sync(stream)
        return ms_

    shapes = {}
    if spp == 2:
        for shp in STEP2_SHAPES:
            h.set_step_blocking(2, ty=shp[0], stages=shp[1], ctas_per_sm=shp[2])
            shapes["ty%d_s%d_c%d" % shp] = g.cells / (timed() / 1e3) / 1e9
        h.set_step_blocking(2)
    ms = timed()
    kernel = h.last_kernel
    val = g.cells / (ms / 1e3) / 1e9
    es = 4 if dtype == "f32" else 2
    bpcs = 6 * es / spp
    peak, kind = measured_peak()
    achieved = bpcs * g.cells / (ms / 1e3) / 1e9
    name = ("step" if spp == 1 else "step2") + ("" if dtype == "f32" else f"-{dtype}")
    extra = {"dtype": dtype, "ms_per_step": ms, "vs_fp32_tend_form": val / ref if ref else None,
             "fp32_tend_gcells": ref,
             "steps_per_pass": spp, "last_kernel": kernel,
             "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                          "frac": achieved / peak, "peak_kind": kind, "bytes_per_cell_step": bpcs},
             "gpu_launches": nsteps // spp + 3}
    if shapes:
        extra["shapes_gcell_steps"] = shapes
    _form_line(args, name,
               f"PW fused forward-Euler step, Gcell-steps/s, {dtype.upper()} state, {spp} step(s) per pass", val,
               "Gcell-steps/s",
               {"workload": f"{nx}x{ny}x{nz} smooth field (w = 0 initially), {nsteps} fused steps per call "
                            f"(dt = 0 keeps the state fixed for timing), halo {spp}", "scales": list(sc)},
               extra)


def form_batch(args, dtype="f32", rank=0, world=1):
    """The batch of independent grids; under torchrun the grids are split
    whole across the ranks (shard.assign_grids, no collective on the data
    path), every rank marches its share in one batched launch, and the job is
    timed by the slowest rank (strong scaling: the batch is fixed)."""
    import paper_2301_13016_gb300 as pwlib
    from paper_2301_13016_gb300 import autotune, inputs, shard
    stream = torch.cuda.current_stream()
    ref = None if (args.skip_fp32_ref or rank != 0) else _fp32_reference_rate(2048, 2048, 64, 50, stream)
    shapes = inputs.batch_shapes(n=args.batch_grids)
    total_cells = sum(nx * ny * nz for nx, ny, nz in shapes)
    mine = shard.assign_grids([nx * ny * nz for nx, ny, nz in shapes], world)[rank]
    grids, coeffs, dev, outs = [], [], [], []
    for q in mine:
        nx, ny, nz = shapes[q]
        g = pwlib.Grid(nx, ny, nz, dtype=dtype)
        c = inputs.make_coeffs(nz)
        d = inputs.random_fields(nx, ny, nz, device="cuda", seeds=(10 + 3 * q, 11 + 3 * q, 12 + 3 * q))
        grids.append(g)
        coeffs.append(c)
        dev.append([g.from_dense(x) for x in d])
        outs.append([g.alloc(fill=None) for _ in range(3)])
        del d
    b = pwlib.Batch(grids, coeffs)
    flds = ([x[0] for x in dev], [x[1] for x in dev], [x[2] for x in dev],
            [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs])
    t0 = time.perf_counter()
    if args.batch_tile:
        v = [int(x) for x in args.batch_tile.split(",")]
        cfg, times = dict(lanes_x=v[0], ty=v[1], stages=v[2], ctas_per_sm=v[3], rows=v[4] if len(v) > 4 else 0,
                          cells=v[5] if len(v) > 5 else 0), {}
        b.set_config(**cfg)
    else:
        cfg, times = autotune.tune_batch(b, flds, reps=3, force=True)
    tune_s = time.perf_counter() - t0
    f = lambda: b.tendencies(*flds, stream=stream)
    for _ in range(args.warmup):
        f()
    b.sync(stream)
    barrier(world)
    torch.cuda.synchronize()
    ms_own = _events_ms(f, args.steps, stream)
    torch.cuda.synchronize()
    barrier(world)
    b.sync(stream)
    ms = max_over_ranks(ms_own, world)
    info = b.info()
    assert info["cells"] == sum(g.cells for g in grids)
    if rank != 0:
        return
    val = total_cells / (ms / 1e3) / 1e9
    peak, kind = measured_peak()
    bpc = 24 if dtype == "f32" else 12
    achieved = bpc * total_cells / (ms / 1e3) / 1e9
    n = args.batch_grids
    name = "batch" if dtype == "f32" else f"batch-{dtype}"
    extra = {"dtype": dtype, "ms_per_step": ms, "vs_fp32_form": val / ref if ref else None, "fp32_form_gcells": ref,
             "autotune_s": tune_s, "autotune_ms": times,
             "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak * world, "unit": "GB/s",
                          "frac": achieved / (peak * world), "peak_kind": kind, "bytes_per_cell": bpc},
             "gpu_launches": args.steps}
    if world > 1:
        extra.update({"n_gpus": world, "scaling": "strong", "rank0_grids": len(mine), "rank0_cells": info["cells"]})
    _form_line(args, name, f"PW tendencies Gcell/s, {n} independent grids in one persistent graph-replayed launch",
               val, "Gcell/s", {"workload": f"{n} grids, nx, ny ~ U{{32..384 step 4}}, nz ~ U{{32..128}} (seed 2304), "
                                            f"{dtype.upper()} storage, FP32 math, random 10*N(0,1)",
                                "cells": total_cells, "items": info["items"], "ctas": info["ctas"], "tile": cfg,
                                "narrow_last_columns": b.narrow_shape(),
                                "parallelism": f"{n} grids split whole over {world} GPU(s)"},
               extra)


def form_adjoint(args):
    import paper_2301_13016_gb300 as pwlib
    from paper_2301_13016_gb300 import inputs
    from paper_2301_13016_gb300.autograd import rollout
    nx = ny = 512
    nz = 64
    nsteps, every, dt = 20, 5, 1.0
    stream = torch.cuda.current_stream()
    ref = None if args.skip_fp32_ref else _fp32_reference_rate(nx, ny, nz, 50, stream)
    c = inputs.make_coeffs(nz)
    g = pwlib.Grid(nx, ny, nz)
    h = pwlib.PW(g, c)
    f = inputs.smooth_fields(nx, ny, nz, w_zero=True, device="cuda")
    ut = inputs.target_field(nx, ny, nz, device="cuda")
    q0 = [g.from_dense(x).requires_grad_(True) for x in f]

    def run():
        for t in q0:
            t.grad = None
        uT, vT, wT = rollout(*q0, h, dt, nsteps, every)
        d = g.view(uT)[1:-1, 1:-1, 1:-1].double() - ut[1:-1, 1:-1, 1:-1].double()
        L = 0.5 * (d * d).sum()
        L.backward()
        return L

    run()
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    reps = max(1, min(args.steps, 5))
    fwd_ms = bwd_ms = 0.0
    for _ in range(reps):
        for t in q0:
            t.grad = None
        e[0].record(stream)
        uT, vT, wT = rollout(*q0, h, dt, nsteps, every)
        d = g.view(uT)[1:-1, 1:-1, 1:-1].double() - ut[1:-1, 1:-1, 1:-1].double()
        L = 0.5 * (d * d).sum()
        e[1].record(stream)
        L.backward()
        e[2].record(stream)
        e[2].synchronize()
        fwd_ms += e[0].elapsed_time(e[1]) / reps
        bwd_ms += e[1].elapsed_time(e[2]) / reps
    # the adjoint kernel alone (one reverse step)
    gs = [g.from_dense(inputs.target_field(nx, ny, nz, std=1.0, seed=2306 + n, device="cuda")) for n in range(3)]
    g2 = [g.alloc() for _ in range(3)]
    qs = [t.detach().clone() for t in q0]
    h.step(*qs, *g2, dt, 0)
    adj = lambda: h.adjoint(*qs, *gs, *g2, alpha=dt, flags=pwlib.PW_ADJ_PERIODIC | pwlib.PW_ADJ_ADD_LAMBDA,
                            stream=stream)
    adj()
    adj_kernel = {1: "adjoint_gather_kernel", 2: "adjoint_vec_kernel"}.get(h.last_kernel, "none")
    adj_ms = _events_ms(adj, 20, stream)
    cell_steps = g.cells * nsteps
    peak, kind = measured_peak()
    adj_gbs = 36 * g.cells / (adj_ms / 1e3) / 1e9
    _form_line(args, "adjoint", "PW adjoint rollout: Gcell-steps/s of forward + backward (checkpointed)",
               cell_steps / ((fwd_ms + bwd_ms) / 1e3) / 1e9, "Gcell-steps/s",
               {"workload": f"{nx}x{ny}x{nz} FP32, {nsteps} Euler steps dt = {dt}, checkpoint every {every}, "
                            "loss 0.5*sum((u_T - u_target)^2), u_target ~ N(0, 10^2) (seed 2305)"},
               {"dtype": "f32", "forward_ms": fwd_ms, "backward_ms": bwd_ms,
                "backward_gcell_steps": cell_steps / (bwd_ms / 1e3) / 1e9,
                "adjoint_kernel_ms": adj_ms, "adjoint_kernel_gcells": g.cells / (adj_ms / 1e3) / 1e9,
                "vs_fp32_form": (g.cells / (adj_ms / 1e3) / 1e9) / ref if ref else None, "fp32_form_gcells": ref,
                "roofline": {"bound": "hbm", "kernel": adj_kernel, "achieved": adj_gbs, "peak": peak,
                             "unit": "GB/s", "frac": adj_gbs / peak, "peak_kind": kind, "bytes_per_cell": 36}})


def form_latency64(args):
    import paper_2301_13016_gb300 as pwlib
    from paper_2301_13016_gb300 import inputs
    nx = ny = nz = 64
    c = inputs.make_coeffs(nz)
    g = pwlib.Grid(nx, ny, nz)
    h = pwlib.PW(g, c)
    dev = [g.from_dense(x) for x in inputs.random_fields(nx, ny, nz)]
    outs = [g.alloc() for _ in range(3)]
    s = torch.cuda.Stream()
    res = {}
    for lx, ty, nseg in ((0, 0, 0), (32, 4, 8), (16, 4, 8), (32, 4, 16), (16, 4, 16), (32, 8, 16), (32, 4, 32),
                         (16, 4, 32)):
        h.set_tma_config(ty, 4 if ty else 0, nseg, lanes_x=lx)   # (0, 0, 0): the automatic shape
        lx, ty = h.tma_config()["lanes_x"], h.tma_config()["ty"]
        with torch.cuda.stream(s):
            for _ in range(3):
                h.tendencies(*dev, *outs, stream=s)
        s.synchronize()
        graph = torch.cuda.CUDAGraph()
        n_in = 100
        with torch.cuda.graph(graph, stream=s):
            for _ in range(n_in):
                h.tendencies(*dev, *outs, stream=s)
        graph.replay()
        torch.cuda.synchronize()
        ms = _events_ms(graph.replay, 20, torch.cuda.current_stream()) / n_in
        direct = _events_ms(lambda: h.tendencies(*dev, *outs), 200, torch.cuda.current_stream())
        res[f"lanes{lx}_ty{ty}_nseg{h.tma_config()['nseg']}"] = {"graph_us_per_call": ms * 1e3,
                                                               "stream_us_per_call": direct * 1e3}
    best = min(v["graph_us_per_call"] for v in res.values())
    _form_line(args, "latency64", "PW tendencies latency per call, 64^3 FP32 (graph replay)", best, "us",
               {"workload": "64x64x64 FP32 random 10*N(0,1); L2-resident, launch-bound (not a roofline point)"},
               {"dtype": "f32", "higher_is_better": False, "shapes": res, "gcells_at_best": g.cells / best / 1e3})


def _torch_cudart():
    """The CUDA runtime library torch loaded (pitched copies, which torch
    does not expose, are issued through it on torch's streams), or None."""
    import ctypes
    torch.cuda.init()
    try:
        with open("/proc/self/maps") as fh:
            for line in fh:
                parts = line.split()
                if len(parts) >= 6 and os.path.basename(parts[-1]).startswith("libcudart.so"):
                    return ctypes.CDLL(parts[-1])
    except OSError:
        pass
    return None


def _pitched_box_copies(rt, g, dst, src, i0, ni, j0, nj, chunks, kind, stream):
    """Issue 3D copies of the box i0..i0+ni-1, j0..j0+nj-1 of each level chunk
    (k0, k1) between two flat FP32 allocations of layout g, as the host path
    copies them (cudaMemcpy3DAsync; kind 1 = host to device, 2 = device to
    host)."""
    import ctypes

    class Pos(ctypes.Structure):
        _fields_ = [("x", ctypes.c_size_t), ("y", ctypes.c_size_t), ("z", ctypes.c_size_t)]

    class PPtr(ctypes.Structure):
        _fields_ = [("ptr", ctypes.c_void_p), ("pitch", ctypes.c_size_t), ("xsize", ctypes.c_size_t),
                    ("ysize", ctypes.c_size_t)]

    class Parms(ctypes.Structure):
        _fields_ = [("srcArray", ctypes.c_void_p), ("srcPos", Pos), ("srcPtr", PPtr), ("dstArray", ctypes.c_void_p),
                    ("dstPos", Pos), ("dstPtr", PPtr), ("extent", Pos), ("kind", ctypes.c_int)]

    rows = g.pitch_k // g.pitch_j
    for k0, k1 in chunks:
        off = 4 * (g.origin + k0 * g.pitch_k + j0 * g.pitch_j + i0)
        p = Parms()
        p.srcPtr = PPtr(src.data_ptr() + off, 4 * g.pitch_j, 4 * ni, rows)
        p.dstPtr = PPtr(dst.data_ptr() + off, 4 * g.pitch_j, 4 * ni, rows)
        p.extent = Pos(4 * ni, nj, k1 - k0 + 1)
        p.kind = kind
        if rt.cudaMemcpy3DAsync(ctypes.byref(p), ctypes.c_void_p(stream.cuda_stream)) != 0:
            raise RuntimeError("cudaMemcpy3DAsync failed")


def form_step_slab(args, rank, world):
    """Fused FP32 Euler steps of one 2048 x 2048 x 64 grid split in y slabs
    over the ranks (slab.step_slabs: the step kernel per slab, then the
    y-halo rows exchanged between neighbours; on one rank nothing is
    exchanged).  Strong scaling: the grid is fixed, the job is timed by the
    slowest rank."""
    import paper_2301_13016_gb300 as pwlib
    from paper_2301_13016_gb300 import inputs, slab
    nx = ny = int(args.workload)
    nz = 64
    stream = torch.cuda.current_stream()
    j0, nyr = slab.slab_rows(ny, world, rank)
    c = inputs.make_coeffs(nz)
    g = pwlib.Grid(nx, nyr, nz)
    h = pwlib.PW(g, c)
    full = inputs.smooth_fields(nx, ny, nz, w_zero=True, device="cuda")
    a = [g.from_dense(f[:, j0:j0 + nyr + 2, :]) for f in full]
    del full
    b = [g.alloc() for _ in range(3)]
    ex = slab.HaloExchangeY(world, rank)
    state = [a, b]

    def f():
        out = slab.step_slabs(h, g, state[0], state[1], 0.0, 2, ex, stream=stream)
        if out[0] is not state[0][0]:
            state.reverse()

    for _ in range(max(1, args.warmup)):
        f()
    torch.cuda.synchronize()
    barrier(world)
    ms_own = _events_ms(f, max(1, args.steps // 2), stream) / 2
    barrier(world)
    ms = max_over_ranks(ms_own, world)
    if rank != 0:
        return
    cells = nx * ny * nz
    val = cells / (ms / 1e3) / 1e9
    peak, kind = measured_peak()
    achieved = 24 * cells / (ms / 1e3) / 1e9
    _form_line(args, "step-slab", "PW fused forward-Euler step of one grid split in y slabs, Gcell-steps/s",
               val, "Gcell-steps/s",
               {"workload": f"{nx}x{ny}x{nz} smooth field (w = 0 initially), dt = 0 keeps the state fixed for timing",
                "ranks": world, "rows_per_rank": [slab.slab_rows(ny, world, r)[1] for r in range(world)],
                "parallelism": f"y slabs over {world} GPU(s), one y-halo row exchange per step"},
               {"dtype": "f32", "ms_per_step": ms, "n_gpus": world, "scaling": "strong",
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak * world, "unit": "GB/s",
                             "frac": achieved / (peak * world), "peak_kind": kind, "bytes_per_cell": 24},
                "gpu_launches": 2 * max(1, args.steps // 2)})


def form_hostlink(args):
    """The bound of the end-to-end number: the host link.  Measures the link's
    rate with plain copies of levels 1..nz of three fields between pinned
    host memory and the device (2048 x 2048 x 64 FP32), one direction at a
    time and both at once, and times the host path itself, which moves the
    inputs with their one-cell halo in and the interior of the outputs out,
    pipelined with the kernel; its bound is those bytes at the rate of both
    directions at once."""
    import paper_2301_13016_gb300 as pwlib
    from paper_2301_13016_gb300 import inputs
    nx = ny = 2048
    nz = 64
    g = pwlib.Grid(nx, ny, nz)
    h = pwlib.PW(g, inputs.make_coeffs(nz))
    n = g.alloc_elems
    gen = torch.Generator().manual_seed(2301)
    hin = [torch.randn(n, generator=gen, dtype=torch.float32).pin_memory() for _ in range(3)]
    hout = [torch.zeros(n, dtype=torch.float32).pin_memory() for _ in range(3)]
    din = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    dout = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    lo = g.origin + g.pitch_k + (1 - g.halo) * g.pitch_j + 1 - g.halo
    hi = g.origin + nz * g.pitch_k + (g.ny + g.halo) * g.pitch_j + g.nx + g.halo + 1
    gb = 3 * (hi - lo) * 4 / 1e9                            # each plain copy
    gb_in = 3 * 4 * (nx + 2) * (ny + 2) * nz / 1e9            # what the host path moves
    gb_out = 3 * 4 * nx * ny * nz / 1e9

    def wall(fn, reps):
        fn()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t) / reps

    def h2d():
        with torch.cuda.stream(s_in):
            for q in range(3):
                din[q][lo:hi].copy_(hin[q][lo:hi], non_blocking=True)

    def d2h():
        with torch.cuda.stream(s_out):
            for q in range(3):
                hout[q][lo:hi].copy_(dout[q][lo:hi], non_blocking=True)

    # the same bytes with one copy stream per field (several copy engines)
    s3 = [torch.cuda.Stream() for _ in range(3)]

    def h2d3():
        for q in range(3):
            with torch.cuda.stream(s3[q]):
                din[q][lo:hi].copy_(hin[q][lo:hi], non_blocking=True)

    def d2h3():
        for q in range(3):
            with torch.cuda.stream(s3[q]):
                hout[q][lo:hi].copy_(dout[q][lo:hi], non_blocking=True)

    # the link without copy engines: SM loads from / stores to pinned host
    # memory through a device view of it (unified addressing)
    class _HostView:
        def __init__(self, t):
            self.__cuda_array_interface__ = {"data": (t.data_ptr(), False), "shape": (t.numel(),),
                                             "typestr": "<f4", "version": 3}

    hv_in = [torch.as_tensor(_HostView(t), device="cuda") for t in hin]
    hv_out = [torch.as_tensor(_HostView(t), device="cuda") for t in hout]

    def sm_read():
        for q in range(3):
            torch.add(hv_in[q][lo:hi], 0.0, out=din[q][lo:hi])

    def sm_write():
        for q in range(3):
            torch.add(dout[q][lo:hi], 0.0, out=hv_out[q][lo:hi])

    # the host path's own copies without the kernel: pitched boxes per 4-level
    # chunk (inputs with a one-cell halo in, output interiors out)
    rt = _torch_cudart()
    chunks = [(1 + c * nz // 16, (c + 1) * nz // 16) for c in range(16)]

    def boxes_both():
        for q in range(3):
            _pitched_box_copies(rt, g, din[q], hin[q], 0, nx + 2, 0, ny + 2, chunks, 1, s_in)
            _pitched_box_copies(rt, g, hout[q], dout[q], 1, nx, 1, ny, chunks, 2, s_out)

    s6 = [torch.cuda.Stream() for _ in range(6)]

    def boxes_six_streams():   # one stream per field and direction
        for q in range(3):
            _pitched_box_copies(rt, g, din[q], hin[q], 0, nx + 2, 0, ny + 2, chunks, 1, s6[q])
            _pitched_box_copies(rt, g, hout[q], dout[q], 1, nx, 1, ny, chunks, 2, s6[3 + q])

    reps = max(2, min(args.steps, 10))
    t_in, t_out = wall(h2d, reps), wall(d2h, reps)
    t_both = wall(lambda: (h2d(), d2h()), reps)
    t_boxes = wall(boxes_both, reps) if rt is not None else None
    t_boxes6 = wall(boxes_six_streams, reps) if rt is not None else None
    t_in3, t_out3 = wall(h2d3, reps), wall(d2h3, reps)
    t_smr, t_smw = wall(sm_read, reps), wall(sm_write, reps)
    t_path = wall(lambda: h.tendencies_host(*hin, *hout), reps)

    def path_async(n=4):   # n steps back to back, one wait
        for _ in range(n):
            h.tendencies_host_async(*hin, *hout)
    t_async = wall(path_async, reps) / 4
    val = g.cells / t_path / 1e9
    t_bound = t_boxes if t_boxes is not None else max(gb_in, gb_out) / (gb / t_both)
    _form_line(args, "hostlink", "PW tendencies end to end through host buffers, against the host-link bound", val,
               "Gcell/s", {"workload": f"{nx}x{ny}x{nz} FP32, pinned host buffers, {gb_in:.3f} GB in and "
                                       f"{gb_out:.3f} GB out per call"},
               {"dtype": "f32", "ms_per_step": t_path * 1e3,
                "copy_gbs": {"h2d_alone": gb / t_in, "d2h_alone": gb / t_out, "each_way_both_at_once": gb / t_both,
                             "h2d_three_streams": gb / t_in3, "d2h_three_streams": gb / t_out3,
                             "sm_loads_from_host": gb / t_smr, "sm_stores_to_host": gb / t_smw},
                "plain_copies_gb_each_way": gb, "plain_copies_both_ms": t_both * 1e3,
                "box_copies_both_ms": t_boxes * 1e3 if t_boxes is not None else None,
                "box_copies_gbs_each_way": gb_in / t_boxes if t_boxes is not None else None,
                "box_copies_six_streams_ms": t_boxes6 * 1e3 if t_boxes6 is not None else None,
                "bound_ms": t_bound * 1e3, "bound_gcells": g.cells / t_bound / 1e9,
                "frac_of_link_bound": t_bound / t_path,
                "async_back_to_back_ms_per_step": t_async * 1e3, "async_back_to_back_gcells": g.cells / t_async / 1e9,
                "async_frac_of_link_bound": t_bound / t_async, "h2d_bytes_per_step": int(gb_in * 1e9),
                "d2h_bytes_per_step": int(gb_out * 1e9)})


def main():
    args = parse()
    rank, world, local = dist_init(args)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        elif args.form == "tend":
            run_ours(args, rank, world, local)
        elif args.form in ("batch", "batch-bf16"):
            form_batch(args, "f32" if args.form == "batch" else "bf16", rank, world)
        elif args.form == "step-slab":
            form_step_slab(args, rank, world)
        elif rank == 0:
            {"tend-bf16": lambda: form_tend_lowp(args, "bf16"), "tend-f16": lambda: form_tend_lowp(args, "f16"),
             "step": lambda: form_step(args, "f32"), "step-bf16": lambda: form_step(args, "bf16"),
             "step2": lambda: form_step(args, "f32", 2), "step2-bf16": lambda: form_step(args, "bf16", 2),
             "step2-f16": lambda: form_step(args, "f16", 2),
             "adjoint": lambda: form_adjoint(args), "latency64": lambda: form_latency64(args),
             "hostlink": lambda: form_hostlink(args)}[args.form]()
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
