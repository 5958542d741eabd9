"""Parity of the CUDA tendency path (through the C ABI) with the CPU oracle.

Bar: max|err| / max|ref| <= 1e-5 per field against the FP64 oracle fed the
same FP32 inputs (FP32 arithmetic, fused multiply-adds allowed).  Sizes span
several tiles with ragged tails; full paper-scale grids are checked on
sampled sub-boxes the oracle computes one by one.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2301_13016_gb300 as pwlib
from paper_2301_13016_gb300 import inputs
from gpu_util import NAN, dense_out, interior, rel_errs, run, setup

pytestmark = pytest.mark.gpu
TOL = 1e-5

SHAPES = [(64, 64, 64), (128, 16, 8), (388, 37, 5), (36, 12, 3), (132, 9, 17), (256, 24, 20)]


@pytest.mark.parametrize("shape", SHAPES, ids=[f"{a}x{b}x{c}" for a, b, c in SHAPES])
@pytest.mark.parametrize("kernel", [1, 2], ids=["generic", "tma"])
def test_parity_random(shape, kernel):
    c, f, g, h, dev, outs = setup(*shape)
    h.set_kernel(kernel)
    run(h, dev, outs)
    assert h.last_kernel == kernel
    got = dense_out(g, outs)
    ref64 = oracle.tendencies(*[x.numpy() for x in f], c)
    assert max(rel_errs(got, ref64)) <= TOL
    ref32 = oracle.tendencies(*[x.numpy() for x in f], c, precision="f32")
    assert max(rel_errs(got, [r.astype(np.float64) for r in ref32])) <= TOL


@pytest.mark.parametrize("shape", [(128, 16, 8), (388, 37, 5), (256, 24, 20)], ids=["128", "388", "256"])
@pytest.mark.parametrize("kernel", [1, 2], ids=["generic", "tma"])
def test_parity_anelastic_coefficients(shape, kernel):
    """Anelastic vertical coefficients (tzc1 != tzc2, tzd1 != tzd2), where a
    swapped or mis-indexed vertical coefficient shows; several k segments
    on the TMA kernel."""
    c = inputs.make_coeffs(shape[2], anelastic=True)
    assert np.abs(c.tzc1 - c.tzc2).max() > 0 and np.abs(c.tzd1 - c.tzd2).max() > 0
    c, f, g, h, dev, outs = setup(*shape, coeffs=c)
    h.set_kernel(kernel)
    for nseg in ((0, min(3, shape[2] // 2)) if kernel == 2 else (0,)):
        if kernel == 2:
            h.set_tma_config(nseg=nseg)
        run(h, dev, outs)
        assert h.last_kernel == kernel
        ref64 = oracle.tendencies(*[x.numpy() for x in f], c)
        assert max(rel_errs(dense_out(g, outs), ref64)) <= TOL


@pytest.mark.parametrize("halo", [2, 3])
@pytest.mark.parametrize("kernel", [1, 2], ids=["generic", "tma"])
def test_parity_deeper_halo(halo, kernel):
    """Grids with a deeper lateral halo (room for periodic images): the scheme
    still reads one halo cell, wherever the interior sits in the layout."""
    nx, ny, nz = 132, 21, 9
    g = pwlib.Grid(nx, ny, nz, halo=halo)
    c, f, g, h, dev, outs = setup(nx, ny, nz, grid=g)
    h.set_kernel(kernel)
    run(h, dev, outs)
    assert h.last_kernel == kernel
    ref64 = oracle.tendencies(*[x.numpy() for x in f], c)
    assert max(rel_errs(dense_out(g, outs), ref64)) <= TOL


@pytest.mark.parametrize("shape", [(64, 64, 64), (388, 37, 5), (36, 12, 3)], ids=["64", "388", "36"])
def test_parity_narrow_tiles(shape):
    c, f, g, h, dev, outs = setup(*shape)
    h.set_kernel(2)
    h.set_tma_config(4, 4, 0, lanes_x=16)
    run(h, dev, outs)
    ref64 = oracle.tendencies(*[x.numpy() for x in f], c)
    assert max(rel_errs(dense_out(g, outs), ref64)) <= TOL


@pytest.mark.parametrize("kernel", [1, 2], ids=["generic", "tma"])
def test_parity_smooth(kernel):
    c, f, g, h, dev, outs = setup(64, 64, 64, smooth=True)
    h.set_kernel(kernel)
    run(h, dev, outs)
    ref = oracle.tendencies(*[x.numpy() for x in f], c)
    assert max(rel_errs(dense_out(g, outs), ref)) <= TOL


@pytest.mark.parametrize("shape", [(5, 3, 3), (7, 9, 4), (3, 2, 3), (13, 1, 6), (1, 5, 3)])
def test_odd_shapes_generic(shape):
    c, f, g, h, dev, outs = setup(*shape)
    run(h, dev, outs)
    assert h.last_kernel == 1        # nx not a multiple of 4: the generic kernel
    ref = oracle.tendencies(*[x.numpy() for x in f], c)
    assert max(rel_errs(dense_out(g, outs), ref)) <= TOL


def test_generic_and_tma_agree():
    c, f, g, h, dev, outs = setup(256, 24, 20)
    h.set_kernel(1)
    run(h, dev, outs)
    a = dense_out(g, outs)
    h.set_kernel(2)
    run(h, dev, outs)
    b = dense_out(g, outs)
    for x, y in zip(a, b):
        assert np.abs(interior(x) - interior(y)).max() <= 1e-6 * np.abs(interior(x)).max()


def test_k_segments_bitwise_and_configs_agree():
    c, f, g, h, dev, outs = setup(256, 24, 20)
    h.set_kernel(2)
    results = {}
    for lx, ty, st in ((32, 4, 4), (32, 8, 3), (32, 8, 4), (32, 8, 6), (32, 16, 3), (16, 4, 4), (16, 8, 4)):
        for nseg in (1, 2, 3, 10):
            h.set_tma_config(ty, st, nseg, lanes_x=lx)
            for o in outs:
                o.fill_(NAN)
            run(h, dev, outs)
            results[(lx, ty, st, nseg)] = dense_out(g, outs)
    for (lx, ty, st, nseg), r in results.items():
        base = results[(lx, ty, st, 1)]
        for x, y in zip(r, base):
            assert np.array_equal(x, y, equal_nan=True), (lx, ty, st, nseg)     # same code path per cell
        ref = results[(32, 4, 4, 1)]
        for x, y in zip(r, ref):
            assert np.abs(interior(x) - interior(y)).max() <= 1e-6 * np.abs(interior(y)).max()


@pytest.mark.parametrize("kernel", [1, 2], ids=["generic", "tma"])
def test_output_halo_and_guard_bands_untouched(kernel):
    nx, ny, nz = 132, 10, 6
    c = inputs.make_coeffs(nz)
    f = inputs.random_fields(nx, ny, nz)
    g = pwlib.Grid(nx, ny, nz)
    h = pwlib.PW(g, c)
    guard = 8192
    dev = [g.from_dense(x) for x in f]
    bufs = [torch.full((g.alloc_elems + 2 * guard,), NAN, device="cuda") for _ in range(3)]
    # 16-byte aligned outputs surrounded by NaN guard bands
    outs = [b[guard:guard + g.alloc_elems] for b in bufs]
    h.set_kernel(kernel)
    run(h, dev, outs)
    for b, o in zip(bufs, outs):
        assert torch.isnan(b[:guard]).all() and torch.isnan(b[guard + g.alloc_elems:]).all()
        v = g.view(o)
        assert torch.isfinite(v[1:-1, 1:-1, 1:-1]).all()
        assert torch.isnan(v[0]).all() and torch.isnan(v[-1]).all()
        assert torch.isnan(v[:, 0]).all() and torch.isnan(v[:, -1]).all()
        assert torch.isnan(v[:, :, 0]).all() and torch.isnan(v[:, :, -1]).all()
        # padding between rows is never written either
        mask = torch.ones(g.alloc_elems, dtype=torch.bool, device="cuda")
        idx = g.view(torch.arange(g.alloc_elems, device="cuda"))
        mask[idx[1:-1, 1:-1, 1:-1].reshape(-1)] = False
        assert torch.isnan(o[mask]).all()


@pytest.mark.parametrize("kernel", [1, 2], ids=["generic", "tma"])
def test_zhalo_planes_never_read(kernel):
    nx, ny, nz = 128, 12, 7
    c, f, g, h, dev, outs = setup(nx, ny, nz)
    h.set_kernel(kernel)
    run(h, dev, outs)
    a = dense_out(g, outs)
    fn = [x.clone() for x in f]
    for x in fn:
        x[0] = NAN
        x[nz + 1] = NAN
    dev2 = [g.from_dense(x) for x in fn]
    run(h, dev2, outs)
    b = dense_out(g, outs)
    for x, y in zip(a, b):
        assert np.array_equal(interior(x), interior(y))


def test_nonfinite_input_propagates_like_oracle():
    nx, ny, nz = 128, 8, 6
    c = inputs.make_coeffs(nz)
    f = list(inputs.random_fields(nx, ny, nz))
    f[0][3, 4, 50] = float("inf")
    f[1][2, 5, 7] = NAN
    c, f, g, h, dev, outs = setup(nx, ny, nz, coeffs=c, fields=f)
    run(h, dev, outs)
    got = dense_out(g, outs)
    ref = oracle.tendencies(*[x.numpy() for x in f], c)
    for x, y in zip(got, ref):
        assert np.array_equal(np.isfinite(interior(x)), np.isfinite(interior(y)))
        m = np.isfinite(interior(y))
        assert np.abs(interior(x)[m] - interior(y)[m]).max() <= TOL * np.abs(interior(y)[m]).max()


def test_custom_layout_generic_and_tma():
    nx, ny, nz = 128, 10, 5
    # wider pitch, interior at a 16-byte (not 128-byte) boundary: TMA-eligible
    g = pwlib.Grid(nx, ny, nz, pitch_j=nx + 12, pitch_k=(nx + 12) * (ny + 2) + 8, origin=3)
    c, f, g, h, dev, outs = setup(nx, ny, nz, grid=g)
    ref = oracle.tendencies(*[x.numpy() for x in f], c)
    for kernel in (1, 2):
        h.set_kernel(kernel)
        run(h, dev, outs)
        assert max(rel_errs(dense_out(g, outs), ref)) <= TOL
    # origin not on a granule boundary: generic only
    g2 = pwlib.Grid(nx, ny, nz, pitch_j=nx + 5, pitch_k=(nx + 5) * (ny + 2) + 1, origin=2)
    c, f, g2, h2, dev2, outs2 = setup(nx, ny, nz, grid=g2, fields=f, coeffs=c)
    run(h2, dev2, outs2)
    assert h2.last_kernel == 1
    assert max(rel_errs(dense_out(g2, outs2), ref)) <= TOL
    h2.set_kernel(2)
    with pytest.raises(pwlib.PwError) as e:
        h2.tendencies(*dev2, *outs2)
    assert e.value.status == pwlib.PW_ERR_UNSUPPORTED


def test_tma_rejects_misaligned_pointers():
    nx, ny, nz = 128, 8, 4
    c, f, g, h, dev, outs = setup(nx, ny, nz)
    h.set_kernel(2)
    big = g.alloc()
    shifted = torch.empty(g.alloc_elems + 1, device="cuda")[1:]     # 4-byte offset
    with pytest.raises(pwlib.PwError) as e:
        h.tendencies(shifted, dev[1], dev[2], *outs)
    assert e.value.status == pwlib.PW_ERR_ALIGN
    h.set_kernel(0)
    shifted.copy_(dev[0])
    run(h, [shifted, dev[1], dev[2]], outs)        # automatic choice falls back to generic
    assert h.last_kernel == 1
    del big


def test_aliasing_rejected():
    c, f, g, h, dev, outs = setup(128, 8, 4)
    with pytest.raises(pwlib.PwError) as e:
        h.tendencies(dev[0], dev[1], dev[2], dev[0], outs[1], outs[2])
    assert e.value.status == pwlib.PW_ERR_ARG


@pytest.mark.parametrize("halo", [1, 3])
def test_fill_halo_periodic(halo):
    nx, ny, nz = 36, 10, 4
    g = pwlib.Grid(nx, ny, nz, halo=halo)
    c = inputs.make_coeffs(nz)
    h = pwlib.PW(g, c)
    rng = np.random.default_rng(0)
    t = g.alloc(fill=NAN)
    v = g.view(t)
    core = torch.tensor(rng.normal(size=(nz, ny, nx)), dtype=torch.float32)
    v[1:-1, halo:halo + ny, halo:halo + nx] = core.cuda()
    h.fill_halo_periodic(t)
    h.sync()
    got = v[1:-1].cpu().numpy()
    ref = np.pad(core.numpy(), ((0, 0), (halo, halo), (halo, halo)), mode="wrap")
    assert np.array_equal(got, ref)
    if halo == 1:
        dense = np.full((nz + 2, ny + 2, nx + 2), np.nan)
        dense[1:-1, 1:-1, 1:-1] = core.numpy()
        assert np.array_equal(got, oracle.fill_halo_periodic(dense)[1:-1])
    assert torch.isnan(v[0]).all() and torch.isnan(v[-1]).all()


def test_energy_identity_on_gpu_output():
    """sum_k dz_u sum u*su = 0 (and likewise v, w): the scheme's conservation
    property, evaluated with the library's FP64 reduction on GPU outputs."""
    nx, ny, nz = 256, 64, 32
    c, f, g, h, dev, outs = setup(nx, ny, nz)
    run(h, dev, outs)
    wu = c.rho_u * c.dz_u
    ww = c.rho_w * c.dz_w
    for q, s, wk, k1 in ((dev[0], outs[0], wu, nz), (dev[1], outs[1], wu, nz), (dev[2], outs[2], ww, nz - 1)):
        tot = h.weighted_dot(q, s, wk=wk, k0=2, k1=k1)
        absw = np.abs(wk)
        scale = h.weighted_dot(q, q, wk=absw, k0=2, k1=k1) ** 0.5 * h.weighted_dot(s, s, wk=absw, k0=2, k1=k1) ** 0.5
        assert abs(tot) <= 1e-6 * scale


def test_mirror_antisymmetry_on_gpu():
    nx, ny, nz = 128, 16, 6
    c = inputs.make_coeffs(nz)
    u, v, w = (x.numpy().astype(np.float64) for x in inputs.random_fields(nx, ny, nz))
    N = nx
    iu = np.array([(N - i - 1) % N + 1 for i in range(1, N + 1)])
    ic = np.array([N + 1 - i for i in range(1, N + 1)])
    up, vp, wp = (np.zeros_like(u) for _ in range(3))
    up[1:-1, 1:-1, 1:-1] = -u[1:-1, 1:-1, iu]
    vp[1:-1, 1:-1, 1:-1] = v[1:-1, 1:-1, ic]
    wp[1:-1, 1:-1, 1:-1] = w[1:-1, 1:-1, ic]
    for x in (up, vp, wp):
        inputs.wrap_halo_(x)
    c, _, g, h, dev, outs = setup(nx, ny, nz, coeffs=c, fields=[torch.tensor(x, dtype=torch.float32) for x in (u, v, w)])
    run(h, dev, outs)
    a = dense_out(g, outs)
    devp = [g.from_dense(torch.tensor(x, dtype=torch.float32)) for x in (up, vp, wp)]
    run(h, devp, outs)
    b = dense_out(g, outs)
    sc = max(np.abs(interior(x)).max() for x in a)
    assert np.abs(interior(b[0]) + a[0][1:-1, 1:-1, iu]).max() <= 1e-6 * sc
    assert np.abs(interior(b[1]) - a[1][1:-1, 1:-1, ic]).max() <= 1e-6 * sc
    assert np.abs(interior(b[2]) - a[2][1:-1, 1:-1, ic]).max() <= 1e-6 * sc


@pytest.mark.parametrize("shape,layout", [((256, 20, 9), None), ((128, 16, 64), None), ((36, 8, 5), None),
                                          ((64, 8, 9), (72, 72 * 10 + 8, 3)), ((128, 12, 10), "halo2")],
                         ids=["2chunks", "16chunks", "unpipelined", "level_pitch_not_whole_rows", "halo2"])
def test_host_path_matches_device_path(shape, layout):
    """The host path gives the device path's bits on the interior and leaves
    every other host cell of the outputs as it was (3D box copies, or 2D
    copies per level when a level is not a whole number of rows)."""
    nx, ny, nz = shape
    grid = None
    if layout == "halo2":
        grid = pwlib.Grid(nx, ny, nz, halo=2)
    elif layout:
        pj, pk, origin = layout
        grid = pwlib.Grid(nx, ny, nz, pitch_j=pj, pitch_k=pk, origin=origin)
    c, f, g, h, dev, outs = setup(nx, ny, nz, grid=grid)
    run(h, dev, outs)
    a = dense_out(g, outs)
    hin = [t.cpu().pin_memory() for t in dev]
    hout = [torch.full((g.alloc_elems,), 7.0, dtype=torch.float32).pin_memory() for _ in range(3)]
    h.tendencies_host(*hin, *hout)
    assert h.last_kernel == 2
    b = [g.to_dense(t).numpy() for t in hout]
    for x, y, t in zip(a, b, hout):
        assert np.array_equal(interior(x), interior(y))
        inside = torch.zeros(g.alloc_elems, dtype=torch.bool)
        hh = g.halo
        g.view(inside)[1:-1, hh:hh + ny, hh:hh + nx] = True
        assert torch.all(t[~inside] == 7.0)


@pytest.mark.parametrize("shape", [(256, 20, 64), (36, 8, 5)], ids=["pipelined", "unpipelined"])
def test_host_path_async_calls_back_to_back(shape):
    """Three asynchronous host calls on one handle without waiting, with
    different inputs and outputs, then one sync: each output equals the
    device path's result for its own inputs (the calls share the staging
    buffers; the next call's inputs travel while the last call's outputs come
    back)."""
    nx, ny, nz = shape
    c, f, g, h, dev, outs = setup(nx, ny, nz)
    sets = []
    for seed in (11, 12, 13):
        d = [g.from_dense(x) for x in inputs.random_fields(nx, ny, nz, seeds=(seed, seed + 10, seed + 20))]
        o = [g.alloc(fill=NAN) for _ in range(3)]
        run(h, d, o)
        hin = [t.cpu().pin_memory() for t in d]
        hout = [torch.full((g.alloc_elems,), 7.0, dtype=torch.float32).pin_memory() for _ in range(3)]
        sets.append((dense_out(g, o), hin, hout))
    for _, hin, hout in sets:
        h.tendencies_host_async(*hin, *hout)
    h.sync()
    for ref, hin, hout in sets:
        for x, t in zip(ref, hout):
            assert np.array_equal(interior(x), interior(g.to_dense(t).numpy()))


@pytest.mark.parametrize("shape,kinds", [((36, 8, 5), (0, 0, 0, 0)), ((256, 20, 16), (1, 0, 1, 0))],
                         ids=["unpipelined", "generic_then_pipelined"])
def test_host_path_async_calls_on_different_streams(shape, kinds):
    """Asynchronous host calls on one handle, each on its own stream, without
    waiting in between: the one-launch path (nz < 8, or the generic kernel)
    runs on the caller's stream only, so each call must still be ordered after
    the previous one (they share the staging buffers).  Kinds alternate the
    generic one-launch path with the pipelined TMA path on the same handle.
    Every output equals the oracle for its own inputs."""
    nx, ny, nz = shape
    c = inputs.make_coeffs(nz)
    g = pwlib.Grid(nx, ny, nz)
    h = pwlib.PW(g, c)
    sets = []
    for n, kind in enumerate(kinds):
        seed = 31 + n
        dense = inputs.random_fields(nx, ny, nz, seeds=(seed, seed + 10, seed + 20))
        ref = oracle.tendencies(*[x.numpy() for x in dense], c)
        hin = [g.from_dense(x, device="cpu").pin_memory() for x in dense]
        hout = [torch.full((g.alloc_elems,), 7.0, dtype=torch.float32).pin_memory() for _ in range(3)]
        sets.append((kind, ref, hin, hout, torch.cuda.Stream()))
    for kind, _, hin, hout, s in sets:
        h.set_kernel(kind)
        h.tendencies_host_async(*hin, *hout, stream=s)
    for *_, s in sets:
        h.sync(s)
    torch.cuda.synchronize()
    for kind, ref, hin, hout, s in sets:
        got = [g.to_dense(t).numpy() for t in hout]
        for e in rel_errs(got, ref):
            assert e <= 1e-5


def test_binding_rejects_tensors_on_the_wrong_side():
    """Host tensors never reach a device entry point (the GPU would fault on
    the address) and device tensors never reach the host entry point."""
    c, f, g, h, dev, outs = setup(64, 8, 5)
    cpu = [t.cpu() for t in dev]
    with pytest.raises(ValueError):
        h.tendencies(*cpu, *outs)
    with pytest.raises(ValueError):
        h.step_to(*dev, *[t.cpu() for t in outs], 1.0)
    with pytest.raises(ValueError):
        h.tendencies_host(*dev, *[t.cpu() for t in outs])
    # the C ABI checks too (pinned host memory: device-addressable, so even a
    # missed check could not fault the GPU)
    import ctypes
    pinned = torch.zeros(g.alloc_elems, dtype=torch.float32).pin_memory()
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    L = pwlib.lib()
    assert L.pw_tendencies(h.h, *[P(t) for t in dev], P(outs[0]), P(outs[1]), P(pinned), None,
                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == pwlib.PW_ERR_ARG
    assert "not device memory" in L.pw_last_error().decode()
    assert L.pw_fill_halo_periodic(h.h, P(pinned), None) == pwlib.PW_ERR_ARG
    run(h, dev, outs)     # the handle still works
    h.sync()


def test_error_norms_kernel():
    nx, ny, nz = 128, 12, 8
    c, f, g, h, dev, outs = setup(nx, ny, nz)
    run(h, dev, outs)
    ref = oracle.tendencies(*[x.numpy() for x in f], c)
    got = dense_out(g, outs)
    for o, r, x in zip(outs, ref, got):
        n = h.error_norms(o, r, k0=1, k1=nz)
        d = interior(x) - interior(r)
        assert n[0] == pytest.approx(np.abs(d).max(), rel=1e-12, abs=1e-300)
        assert n[1] == pytest.approx(np.abs(interior(r)).max(), rel=1e-12)
        assert n[2] == pytest.approx(np.sum(d * d), rel=1e-9)
        assert n[3] == pytest.approx(np.sum(interior(r) ** 2), rel=1e-9)


def test_bounded_wait_timeout_is_reported_and_context_survives():
    c, f, g, h, dev, outs = setup(128, 8, 5)
    h.selftest_wait_timeout(50_000_000)
    with pytest.raises(pwlib.PwError) as e:
        h.sync()
    assert e.value.status == pwlib.PW_ERR_DEVICE_TIMEOUT
    h.sync()          # cleared
    run(h, dev, outs)
    ref = oracle.tendencies(*[x.numpy() for x in f], c)
    assert max(rel_errs(dense_out(g, outs), ref)) <= TOL


def _subbox(f, j0, i0, n):
    """Dense sub-array with one halo cell around interior rows j0..j0+n-1 and
    columns i0..i0+n-1 (all levels)."""
    return f[:, j0 - 1:j0 + n + 1, i0 - 1:i0 + n + 1]


def test_full_512_parity():
    nx = ny = 512
    nz = 64
    for smooth in (False, True):
        c, f, g, h, dev, outs = setup(nx, ny, nz, smooth=smooth)
        run(h, dev, outs)
        assert h.last_kernel == 2
        ref = oracle.tendencies(*[x.numpy() for x in f], c)
        assert max(rel_errs(dense_out(g, outs), ref)) <= TOL


def test_sampled_parity_2048():
    """The paper-scale grid 2048 x 2048 x 64 in the benchmark's launch shape,
    checked on sampled 32 x 32 column boxes (edges, corners, interior)."""
    nx = ny = 2048
    nz = 64
    c = inputs.make_coeffs(nz)
    f = inputs.random_fields(nx, ny, nz, device="cuda")
    g = pwlib.Grid(nx, ny, nz)
    h = pwlib.PW(g, c)
    dev = [g.from_dense(x) for x in f]
    outs = [g.alloc(fill=NAN) for _ in range(3)]
    run(h, dev, outs)
    assert h.last_kernel == 2
    n = 32
    rng = np.random.default_rng(1)
    corners = [(1, 1), (1, nx - n + 1), (ny - n + 1, 1), (ny - n + 1, nx - n + 1)]
    corners += [(int(rng.integers(1, ny - n)), int(rng.integers(1, nx - n))) for _ in range(4)]
    views = [g.view(o) for o in outs]
    for j0, i0 in corners:
        sub = [_subbox(x, j0, i0, n).cpu().numpy() for x in f]
        ref = oracle.tendencies(*sub, c)
        got = [_subbox(v, j0, i0, n).cpu().double().numpy() for v in views]
        errs = rel_errs(got, ref)
        assert max(errs) <= TOL, (j0, i0, errs)
