"""The N > 1 path of bench.py on CPU: two ranks over the gloo backend
(127.0.0.1), no GPU.  The path shards by independent grids with no data-path
collective; what is shared is the host logic: rank setup from the torchrun
environment, the barrier and the max over ranks that time the job, the
weak-scaling rate, and the reference arm, which rank 0 alone runs and prints.
"""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _Args:
    impl = "reference"


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    r, w, _ = bench.dist_init(_Args)
    assert dist.get_backend() == "gloo"
    slowest = bench.max_over_ranks(0.5 + rank, w)   # rank 1 is the slower one
    bench.barrier(w)
    q.put((r, w, slowest, bench.whole_job_rate(1000, w, slowest)))
    dist.destroy_process_group()


def test_two_ranks_time_the_job_by_the_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    for _, world, slowest, rate in got:
        assert world == 2 and slowest == 1.5
        assert rate == 1000 * 2 / 1.5


def test_reference_arm_under_torchrun_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--workload", "512"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def _assign_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    from paper_2301_13016_gb300 import inputs, shard
    bench.dist_init(_Args)
    sizes = [nx * ny * nz for nx, ny, nz in inputs.batch_shapes()]
    mine = shard.assign_grids(sizes, world)[rank]
    got = [None] * world
    dist.all_gather_object(got, mine)   # test only: the ranks never exchange this in the bench
    q.put((rank, got))
    dist.destroy_process_group()


def test_batch_grids_split_whole_over_ranks():
    """Every rank derives the same whole-grid assignment of the 512-grid batch
    from the sizes alone: the ranks' lists are disjoint, cover every grid, and
    the largest load exceeds the mean by less than one grid."""
    from paper_2301_13016_gb300 import inputs, shard
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_assign_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    views = [g for _, g in got]
    assert views[0] == views[1]                       # one assignment, derived independently
    lists = views[0]
    sizes = [nx * ny * nz for nx, ny, nz in inputs.batch_shapes()]
    assert sorted(i for l in lists for i in l) == list(range(len(sizes)))
    loads = [sum(sizes[i] for i in l) for l in lists]
    assert max(loads) - sum(sizes) / 2 < max(sizes)
    for world in (1, 3, 4, 8):
        a = shard.assign_grids(sizes, world)
        assert sorted(i for l in a for i in l) == list(range(len(sizes)))
        ld = [sum(sizes[i] for i in l) for l in a]
        assert max(ld) - sum(sizes) / world < max(sizes)
    assert shard.assign_grids([5, 1, 1, 1], 2) == [[0], [1, 2, 3]]


def _slab_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2301_13016_gb300 import inputs, slab
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nx, ny, nz, dt, nsteps = 12, 11, 6, 2.0, 5
    c = inputs.make_coeffs(nz)
    full = [f.double() for f in inputs.smooth_fields(nx, ny, nz)]        # periodic halos filled
    j0, nyr = slab.slab_rows(ny, world, rank)
    mine = [f[:, j0:j0 + nyr + 2, :].clone() for f in full]             # the slab with its halo rows
    ex = slab.HaloExchangeY(world, rank)
    for _ in range(nsteps):
        # the local step: the oracle's source terms of the slab as it stands,
        # the update, the x images; then the y-halo rows from the neighbours
        s = oracle.tendencies(*[m.numpy() for m in mine], c)
        for m, sm in zip(mine, s):
            m[1:-1, 1:-1, 1:-1] += dt * torch.from_numpy(sm)[1:-1, 1:-1, 1:-1]
            m[:, 1:-1, 0] = m[:, 1:-1, nx]
            m[:, 1:-1, nx + 1] = m[:, 1:-1, 1]
        ex.exchange(mine)
    q.put((rank, j0, nyr, [m.numpy() for m in mine]))
    dist.destroy_process_group()


def test_slab_decomposed_steps_match_the_undivided_grid():
    """Five Euler steps of one grid split in y over 2 and 3 gloo ranks (the
    oracle's source terms per slab, the library's halo exchange between
    them) give the undivided grid's oracle steps, halo rows included."""
    import numpy as np
    import oracle
    from paper_2301_13016_gb300 import inputs, slab
    nx, ny, nz, dt, nsteps = 12, 11, 6, 2.0, 5
    c = inputs.make_coeffs(nz)
    ref = oracle.step(*[f.double().numpy() for f in inputs.smooth_fields(nx, ny, nz)], c, dt, nsteps)
    for world in (2, 3):
        ctx = mp.get_context("spawn")
        q = ctx.Queue()
        port = _free_port()
        procs = [ctx.Process(target=_slab_main, args=(r, world, port, q)) for r in range(world)]
        for p in procs:
            p.start()
        got = sorted((q.get(timeout=180) for _ in procs), key=lambda t: t[0])
        for p in procs:
            p.join(timeout=60)
            assert p.exitcode == 0
        assert [g[1] for g in got] == [slab.slab_rows(ny, world, r)[0] for r in range(world)]
        assert sum(g[2] for g in got) == ny
        for f in range(3):
            for rank, j0, nyr, arrs in got:
                a = arrs[f][1:-1, :, :]                          # levels 1..nz, halo rows and columns
                r = ref[f][1:-1, j0:j0 + nyr + 2, :]
                assert np.allclose(a, r, rtol=1e-12, atol=1e-12 * np.abs(ref[f]).max())
    assert slab.slab_rows(10, 3, 0) == (0, 4) and slab.slab_rows(10, 3, 2) == (7, 3)
