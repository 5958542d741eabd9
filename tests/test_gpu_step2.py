"""Two forward-Euler steps per kernel pass (temporal blocking) through the C
ABI.

FP32 storage: the two-step pass runs the same per-level arithmetic as the
single-step pass and keeps the intermediate state in FP32, so the result must
equal two single-step passes BIT FOR BIT, halos included; and it is checked
against the FP64 oracle rollout (oracle.step) with the single-step bar
(max|err| / max|ref| <= 1e-5 per step).  Covered: every instantiated launch
shape, ragged tiles in x and y (tiles are 120 x (ty-2) outputs), several k
segments, odd step counts (a single-step pass finishes them), the shallowest
grids (nz = 3) and a deeper halo.

16-bit storage: the intermediate state is not rounded to the storage type,
so the two-step result differs from two single-step passes; it is checked
against the FP64 oracle with the 16-bit bars of the single-step tests.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2301_13016_gb300 as pwlib
from paper_2301_13016_gb300 import inputs, precision
from gpu_util import NAN, interior

pytestmark = pytest.mark.gpu

SHAPES = [(8, 3, 1), (8, 3, 2), (8, 4, 1), (12, 3, 1), (16, 3, 1), (16, 4, 1)]


def _fields(nx, ny, nz, smooth):
    return inputs.smooth_fields(nx, ny, nz) if smooth else inputs.random_fields(nx, ny, nz)


def _run(g, c, f, nsteps, dt, spp, shape=None, nseg=0, scale=None):
    """Fresh handle and buffers; returns (state tensors, handle)."""
    h = pwlib.PW(g, c)
    ty, st, cps = shape if shape else (0, 0, 0)
    h.set_step_blocking(spp, ty=ty, stages=st, ctas_per_sm=cps, nseg=nseg)
    q = [g.from_dense(x, scale=s) for x, s in zip(f, scale or (1.0, 1.0, 1.0))]
    for t in q:   # garbage halos: pw_step refreshes them itself
        v = g.view(t)
        v[1:-1, 0] = NAN
        v[1:-1, :, -1] = NAN
    tmp = [g.alloc(fill=NAN) for _ in range(3)]
    h.step(*q, *tmp, dt, nsteps, scale=scale)
    h.sync()
    return q, h


def _levels(g, t):
    """levels 1..nz of a field, lateral halo included"""
    return g.view(t)[1:-1]


def _relerr(got, ref):
    return max(float(np.abs(interior(a) - interior(b)).max() / np.abs(interior(b)).max())
               for a, b in zip(got, ref) if np.abs(interior(b)).max() > 0)


@pytest.mark.parametrize("shape", SHAPES, ids=[f"ty{a}_s{b}_c{c}" for a, b, c in SHAPES])
@pytest.mark.parametrize("dims,nsteps,smooth", [((128, 24, 16), 2, True), ((388, 13, 7), 4, False),
                                                ((364, 29, 3), 3, False), ((8, 2, 5), 2, False)])
def test_two_step_equals_single_steps_bitwise(shape, dims, nsteps, smooth):
    nx, ny, nz = dims
    c = inputs.make_coeffs(nz)
    f = _fields(nx, ny, nz, smooth)
    g = pwlib.Grid(nx, ny, nz, halo=2)
    q2, h2 = _run(g, c, f, nsteps, 0.5, 2, shape)
    q1, h1 = _run(g, c, f, nsteps, 0.5, 1)
    assert h2.last_kernel == 3 and h1.last_kernel == 2
    for a, b in zip(q2, q1):
        assert torch.equal(_levels(g, a), _levels(g, b))
    ref = oracle.step(*[x.numpy() for x in f], c, 0.5, nsteps)
    got = [g.to_dense(t).numpy() for t in q2]
    assert _relerr(got, ref) <= 1e-5 * nsteps
    for x in got:   # periodic halos of the result at every level 1..nz
        assert np.array_equal(x[1:-1], oracle.fill_halo_periodic(x)[1:-1])


@pytest.mark.parametrize("nseg", [2, 3, 8])
def test_two_step_k_segments(nseg):
    nx, ny, nz = 256, 20, 24
    c = inputs.make_coeffs(nz, anelastic=True)
    f = _fields(nx, ny, nz, False)
    g = pwlib.Grid(nx, ny, nz, halo=2)
    q2, h2 = _run(g, c, f, 6, 0.25, 2, nseg=nseg)
    q1, _ = _run(g, c, f, 6, 0.25, 1)
    assert h2.last_kernel == 3
    for a, b in zip(q2, q1):
        assert torch.equal(_levels(g, a), _levels(g, b))


def test_two_step_deep_halo_and_auto_choice():
    nx, ny, nz = 128, 12, 6
    c = inputs.make_coeffs(nz)
    f = _fields(nx, ny, nz, True)
    g = pwlib.Grid(nx, ny, nz, halo=3)
    q0, h0 = _run(g, c, f, 2, 1.0, 0)
    assert h0.last_kernel == 2   # automatic: one step per pass
    q, h = _run(g, c, f, 2, 1.0, 2)
    assert h.last_kernel == 3
    for a, b in zip(q, q0):
        assert torch.equal(_levels(g, a), _levels(g, b))
    ref = oracle.step(*[x.numpy() for x in f], c, 1.0, 2)
    assert _relerr([g.to_dense(t).numpy() for t in q], ref) <= 2e-5
    v = g.view(q[0])[1:-1].cpu().numpy()
    assert np.array_equal(v, np.pad(v[:, 3:-3, 3:-3], ((0, 0), (3, 3), (3, 3)), mode="wrap"))


def test_two_step_full_size_equals_single_steps():
    """2048 x 2048 x 64 FP32, the launch shape the bench times: two-step
    passes equal single-step passes bit for bit on the whole state."""
    nx, ny, nz = 2048, 2048, 64
    c = inputs.make_coeffs(nz)
    f = inputs.random_fields(nx, ny, nz, device="cuda")
    g = pwlib.Grid(nx, ny, nz, halo=2)
    q2, h2 = _run(g, c, f, 2, 1.0, 2)
    q1, _ = _run(g, c, f, 2, 1.0, 1)
    assert h2.last_kernel == 3
    for a, b in zip(q2, q1):
        assert torch.equal(_levels(g, a), _levels(g, b))
    del q1, q2
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype,bound", [("bf16", 0.05), ("f16", 0.01)])
def test_two_step_lowp_state(dtype, bound):
    """16-bit state, 10 steps (5 two-step passes) on the smooth field with
    w = 0 initially, against the FP64 rollout of the original FP32 fields."""
    nx, ny, nz = 128, 32, 16
    c = inputs.make_coeffs(nz)
    f = inputs.smooth_fields(nx, ny, nz, w_zero=True)
    maxabs = [max(float(x.abs().max()), 1.0) for x in f]
    sc = precision.suggest_scales(maxabs, c, dtype)[:3]
    g = pwlib.Grid(nx, ny, nz, dtype=dtype, halo=2)
    ref = oracle.step(*[x.numpy() for x in f], c, 1.0, 10)
    errs = {}
    for spp in (2, 1):
        q, h = _run(g, c, f, 10, 1.0, spp, scale=sc)
        assert h.last_kernel == (3 if spp == 2 else 2)
        got = [g.to_dense(t, s).numpy() for t, s in zip(q, sc)]
        e = [float(np.abs(interior(a) - interior(b)).max() / np.abs(interior(b)).max())
             for a, b in zip(got[:2], ref[:2])]
        e.append(float(np.abs(interior(got[2]) - interior(ref[2])).max() / np.abs(interior(ref[0])).max()))
        errs[spp] = max(e)
    assert errs[2] <= bound
    # half as many roundings of the state: not worse than one step per pass
    assert errs[2] <= 1.1 * errs[1], errs


def test_two_step_requirements():
    nx, ny, nz = 128, 8, 5
    c = inputs.make_coeffs(nz)
    f = _fields(nx, ny, nz, False)
    g1 = pwlib.Grid(nx, ny, nz)   # halo 1
    h = pwlib.PW(g1, c)
    h.set_step_blocking(2)
    q = [g1.from_dense(x) for x in f]
    tmp = [g1.alloc() for _ in range(3)]
    with pytest.raises(pwlib.PwError) as e:
        h.step(*q, *tmp, 1.0, 2)
    assert e.value.status == pwlib.PW_ERR_UNSUPPORTED
    h.step(*q, *tmp, 1.0, 1)      # one step needs no two-step pass
    h.set_step_blocking(0)        # automatic: single steps on a halo-1 grid
    h.step(*q, *tmp, 1.0, 2)
    h.sync()
    assert h.last_kernel == 2
    g2 = pwlib.Grid(nx, ny, nz, halo=2)
    h2 = pwlib.PW(g2, c)
    with pytest.raises(pwlib.PwError) as e:
        h2.set_step_blocking(2, ty=10)
    assert e.value.status == pwlib.PW_ERR_UNSUPPORTED
    with pytest.raises(pwlib.PwError) as e:
        h2.set_step_blocking(3)
    assert e.value.status == pwlib.PW_ERR_ARG
    h2.set_kernel(1)              # the generic kernel has no two-step form
    h2.set_step_blocking(2)
    q2 = [g2.from_dense(x) for x in f]
    tmp2 = [g2.alloc() for _ in range(3)]
    with pytest.raises(pwlib.PwError) as e:
        h2.step(*q2, *tmp2, 1.0, 2)
    assert e.value.status == pwlib.PW_ERR_UNSUPPORTED
