"""Autotuner for the k-march launch shapes.

Measures each candidate shape on the caller's own buffers with CUDA events
and keeps the fastest, caching the choice in a JSON file keyed by the grid
shapes, the dtype, the GPU name and its SM count (the cache file is
~/.cache/pw_gb300_tune.json unless a path is given).

  tune_batch(batch, fields)   shape of the persistent batched kernel
                              (lanes per row, rows, stages, CTAs per SM)
  tune_grid(handle, fields)   shape of the single-grid kernel
                              (lanes per row, rows, stages, k segments)
"""
import hashlib
import json
import os

import torch

BATCH_CANDIDATES = [dict(lanes_x=lx, ty=ty, stages=4, ctas_per_sm=c, rows=rp, cells=nc)
                    for lx, ty, nc, rp in ((32, 4, 4, 1), (32, 8, 4, 1), (16, 4, 4, 1), (16, 8, 4, 1), (16, 16, 4, 1),
                                           (32, 8, 4, 2),
                                           (16, 8, 4, 2), (32, 8, 4, 3), (16, 8, 4, 3), (16, 8, 8, 3), (16, 4, 8, 3),
                                           (8, 8, 8, 3), (8, 16, 8, 3), (8, 16, 4, 1), (32, 16, 4, 1))
                    for c in (0, 2)]
GRID_CANDIDATES = [dict(lanes_x=lx, ty=ty, stages=st, nseg=ns, cells=nc, rows=rp)
                   for lx, ty, st, nc, rp in ((32, 4, 4, 4, 1), (32, 8, 4, 4, 1), (32, 8, 6, 4, 1), (16, 4, 4, 4, 1),
                                              (16, 8, 4, 4, 1), (16, 4, 4, 8, 1), (16, 8, 4, 8, 1), (32, 8, 4, 4, 2),
                                              (32, 16, 4, 4, 2), (16, 8, 4, 4, 2), (16, 4, 4, 8, 3),
                                              (16, 8, 4, 8, 3), (16, 16, 4, 8, 3), (32, 4, 4, 4, 3), (32, 8, 4, 4, 3),
                                              (8, 8, 4, 8, 3), (8, 16, 4, 8, 3))
                   for ns in (0, 1, 2, 4)]


def _default_cache():
    return os.path.join(os.path.expanduser("~"), ".cache", "pw_gb300_tune.json")


def _device_key():
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|{p.multi_processor_count}"


def _signature(kind, shapes, dtype):
    h = hashlib.sha256(json.dumps([kind, dtype, shapes]).encode()).hexdigest()[:20]
    return f"{kind}|{dtype}|{_device_key()}|{h}"


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(path, key, value):
    data = _load(path)
    data[key] = value
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time(fn, warmup, reps, stream):
    for _ in range(warmup):
        fn()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_batch(batch, fields, candidates=None, warmup=2, reps=5, cache_path=None, force=False):
    """Pick and apply the fastest batched-kernel shape for `batch`.
    fields = (us, vs, ws, sus, svs, sws), lists of flat device tensors.
    Returns (config, {config string: ms})."""
    cache_path = cache_path or _default_cache()
    shapes = [[g.nx, g.ny, g.nz] for g in batch.grids]
    key = _signature("batch", shapes, batch.grids[0].dtype)
    cached = _load(cache_path).get(key)
    if cached and not force:
        batch.set_config(**cached["config"])
        return cached["config"], cached.get("times", {})
    stream = torch.cuda.current_stream()
    times = {}
    best, best_ms = None, float("inf")
    for c in candidates or BATCH_CANDIDATES:
        try:
            batch.set_config(**c)
        except RuntimeError:
            continue
        ms = _time(lambda: batch.tendencies(*fields, stream=stream), warmup, reps, stream)
        batch.sync(stream)
        times[json.dumps(c, sort_keys=True)] = ms
        if ms < best_ms:
            best, best_ms = c, ms
    if best is None:
        raise RuntimeError("no batched kernel shape could run")
    batch.set_config(**best)
    _store(cache_path, key, {"config": best, "times": times})
    return best, times


def tune_grid(handle, fields, candidates=None, warmup=2, reps=5, cache_path=None, force=False):
    """Pick and apply the fastest single-grid k-march shape for `handle`.
    fields = (u, v, w, su, sv, sw) flat device tensors.  Returns (config, times)."""
    cache_path = cache_path or _default_cache()
    g = handle.grid
    key = _signature("grid", [[g.nx, g.ny, g.nz]], g.dtype)
    cached = _load(cache_path).get(key)
    if cached and not force:
        handle.set_tma_config(**cached["config"])
        return cached["config"], cached.get("times", {})
    stream = torch.cuda.current_stream()
    times = {}
    best, best_ms = None, float("inf")
    for c in candidates or GRID_CANDIDATES:
        if c["nseg"] > g.nz // 2:
            continue
        try:
            handle.set_tma_config(**c)
        except RuntimeError:
            continue
        ms = _time(lambda: handle.tendencies(*fields, stream=stream), warmup, reps, stream)
        handle.sync(stream)
        times[json.dumps(c, sort_keys=True)] = ms
        if ms < best_ms:
            best, best_ms = c, ms
    if best is None:
        raise RuntimeError("no k-march shape could run")
    handle.set_tma_config(**best)
    _store(cache_path, key, {"config": best, "times": times})
    return best, times


def main(argv=None):
    """python -m paper_2301_13016_gb300.autotune NX NY NZ [--dtype f32] [--json]
    Times every single-grid launch shape on a seeded random grid (tendencies
    and fused steps) and prints one JSON line."""
    import argparse
    import paper_2301_13016_gb300 as pwlib
    from paper_2301_13016_gb300 import inputs, precision

    p = argparse.ArgumentParser()
    p.add_argument("nx", type=int)
    p.add_argument("ny", type=int)
    p.add_argument("nz", type=int)
    p.add_argument("--dtype", default="f32", choices=["f32", "bf16", "f16"])
    p.add_argument("--reps", type=int, default=20)
    p.add_argument("--tag", default="")
    p.add_argument("--only", default="", help="one shape LANES,TY,STAGES,CELLS[,ROWS] (e.g. 16,8,4,8)")
    a = p.parse_args(argv)
    only = tuple(int(x) for x in a.only.split(",")) if a.only else None
    c = inputs.make_coeffs(a.nz)
    g = pwlib.Grid(a.nx, a.ny, a.nz, dtype=a.dtype)
    h = pwlib.PW(g, c)
    dense = inputs.random_fields(a.nx, a.ny, a.nz, device="cuda")
    sc = precision.suggest_scales([float(x.abs().max()) for x in dense], c, a.dtype)
    dev = [g.from_dense(x, scale=s) for x, s in zip(dense, sc[:3])]
    del dense
    outs = [g.alloc() for _ in range(3)]
    tmp = [g.alloc() for _ in range(3)]
    stream = torch.cuda.current_stream()
    res = {}
    seen = set()
    for cand in GRID_CANDIDATES:
        key = (cand["lanes_x"], cand["ty"], cand["stages"], cand["cells"], cand["rows"])
        if key in seen or (only and key[:len(only)] != only):
            continue
        seen.add(key)
        try:
            h.set_tma_config(cand["ty"], cand["stages"], 0, lanes_x=cand["lanes_x"], cells=cand["cells"],
                             rows=cand["rows"])
        except RuntimeError:
            continue
        ms_t = _time(lambda: h.tendencies(*dev, *outs, scale=sc, stream=stream), 3, a.reps, stream)
        ms_s = _time(lambda: h.step(*dev, *tmp, 0.0, 2, scale=sc[:3], stream=stream), 2, a.reps, stream) / 2
        h.sync(stream)
        res[f"lanes{key[0]}_ty{key[1]}_s{key[2]}_c{key[3]}_r{key[4]}"] = {"tend_gcells": g.cells / ms_t / 1e6,
                                                      "step_gcells": g.cells / ms_s / 1e6}
    print(json.dumps({"grid": [a.nx, a.ny, a.nz], "dtype": a.dtype, "tag": a.tag, "device": _device_key(),
                      "shapes": res}), flush=True)


if __name__ == "__main__":
    main()
