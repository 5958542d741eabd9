"""pw_step (fused forward-Euler steps) through the C ABI against the FP64
oracle's rollout (oracle.step: fill halo, tendencies, update, per step).

FP32 state: the per-step rounding of the state and the FP32 source terms
give a relative error that grows about linearly with the step count; the
bar is max|err| / max|ref| <= 1e-5 per step taken.  16-bit state: the state
is rounded to the storage type every step; bars stated per format below.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2301_13016_gb300 as pwlib
from paper_2301_13016_gb300 import inputs, precision
from gpu_util import NAN, interior

pytestmark = pytest.mark.gpu


def _state(nx, ny, nz, smooth=True, w_zero=False, dtype="f32", grid=None, scale=(1.0, 1.0, 1.0)):
    c = inputs.make_coeffs(nz)
    f = inputs.smooth_fields(nx, ny, nz, w_zero=w_zero) if smooth else inputs.random_fields(nx, ny, nz)
    g = grid if grid is not None else pwlib.Grid(nx, ny, nz, dtype=dtype)
    h = pwlib.PW(g, c)
    q = [g.from_dense(x, scale=s) for x, s in zip(f, scale)]
    for t in q:               # garbage halos: pw_step must refresh them itself
        v = g.view(t)
        v[1:-1, 0] = NAN
        v[1:-1, :, 0] = NAN
    tmp = [g.alloc(fill=NAN) for _ in range(3)]
    return c, f, g, h, q, tmp


def _dense(g, q, scale=(1.0, 1.0, 1.0)):
    return [g.to_dense(t, s).numpy() for t, s in zip(q, scale)]


def _relerr(got, ref):
    return max(float(np.abs(interior(a) - interior(b)).max() / np.abs(interior(b)).max())
               for a, b in zip(got, ref) if np.abs(interior(b)).max() > 0)


@pytest.mark.parametrize("kernel", [1, 2], ids=["generic", "tma"])
def test_step_anelastic_matches_oracle_rollout(kernel):
    """Anelastic vertical coefficients through the fused step (3 steps)."""
    nx, ny, nz = 128, 24, 16
    c, f, g, h, q, tmp = _state(nx, ny, nz)
    c = inputs.make_coeffs(nz, anelastic=True)
    h = pwlib.PW(g, c)
    h.set_kernel(kernel)
    h.step(*q, *tmp, 1.0, 3)
    h.sync()
    assert h.last_kernel == kernel
    ref = oracle.step(*[x.numpy() for x in f], c, 1.0, 3)
    assert _relerr(_dense(g, q), ref) <= 3e-5


@pytest.mark.parametrize("kernel", [1, 2], ids=["generic", "tma"])
@pytest.mark.parametrize("nsteps", [1, 2, 5])
def test_step_matches_oracle_rollout(kernel, nsteps):
    nx, ny, nz = 128, 24, 16
    c, f, g, h, q, tmp = _state(nx, ny, nz)
    h.set_kernel(kernel)
    dt = 1.0
    h.step(*q, *tmp, dt, nsteps)
    h.sync()
    assert h.last_kernel == kernel
    got = _dense(g, q)
    ref = oracle.step(*[x.numpy() for x in f], c, dt, nsteps)
    assert _relerr(got, ref) <= 1e-5 * nsteps
    # halos of the result are the periodic images, at every level 1..nz
    for x in got:
        assert np.array_equal(x[1:-1], oracle.fill_halo_periodic(x)[1:-1])


def test_step_random_fields_and_ragged_tiles():
    nx, ny, nz = 388, 13, 7
    c, f, g, h, q, tmp = _state(nx, ny, nz, smooth=False)
    h.step(*q, *tmp, 0.25, 3)
    h.sync()
    assert h.last_kernel == 2
    ref = oracle.step(*[x.numpy() for x in f], c, 0.25, 3)
    assert _relerr(_dense(g, q), ref) <= 3e-5


@pytest.mark.parametrize("shape,kernel", [((5, 3, 3), 1), ((12, 1, 4), 1), ((12, 1, 4), 2), ((1, 6, 5), 1),
                                          ((4, 4, 3), 2), ((4, 1, 3), 2)])
def test_step_odd_shapes(shape, kernel):
    c, f, g, h, q, tmp = _state(*shape, smooth=False)
    h.set_kernel(kernel)
    h.step(*q, *tmp, 0.5, 2)
    h.sync()
    assert h.last_kernel == kernel
    ref = oracle.step(*[x.numpy() for x in f], c, 0.5, 2)
    got = _dense(g, q)
    assert _relerr(got, ref) <= 2e-5
    for x in got:
        assert np.array_equal(x[1:-1], oracle.fill_halo_periodic(x)[1:-1])


def test_step_deep_halo_layout():
    nx, ny, nz = 128, 12, 6
    g = pwlib.Grid(nx, ny, nz, halo=3)
    c, f, g, h, q, tmp = _state(nx, ny, nz, grid=g)
    h.step(*q, *tmp, 1.0, 2)
    h.sync()
    ref = oracle.step(*[x.numpy() for x in f], c, 1.0, 2)
    assert _relerr(_dense(g, q), ref) <= 2e-5
    v = g.view(q[0])[1:-1].cpu().numpy()
    assert np.array_equal(v, np.pad(v[:, 3:-3, 3:-3], ((0, 0), (3, 3), (3, 3)), mode="wrap"))


def test_step_zero_steps_refreshes_halo_only():
    c, f, g, h, q, tmp = _state(128, 8, 5)
    before = [g.view(t)[1:-1, 1:-1, 1:-1].clone() for t in q]
    h.step(*q, *tmp, 1.0, 0)
    h.sync()
    for t, b in zip(q, before):
        assert torch.equal(g.view(t)[1:-1, 1:-1, 1:-1], b)
    for x in _dense(g, q):
        assert np.array_equal(x[1:-1], oracle.fill_halo_periodic(x)[1:-1])


def test_step_energy_growth_matches_euler_identity():
    """||q_{n+1}||_W^2 - ||q_n||_W^2 = dt^2 ||s(q_n)||_W^2 (Euler + the scheme's
    energy identity), with W the level weights, on the GPU state."""
    nx, ny, nz = 256, 32, 16
    c, f, g, h, q, tmp = _state(nx, ny, nz, smooth=False)
    for t in q:
        h.fill_halo_periodic(t)
    s = [g.alloc() for _ in range(3)]
    h.tendencies(*q, *s)
    wu, ww = c.rho_u * c.dz_u, c.rho_w * c.dz_w
    dt = 0.5

    def energy(fields):
        return (h.weighted_dot(fields[0], fields[0], wk=wu, k0=2, k1=nz) +
                h.weighted_dot(fields[1], fields[1], wk=wu, k0=2, k1=nz) +
                h.weighted_dot(fields[2], fields[2], wk=ww, k0=2, k1=nz - 1))

    e0 = energy(q)
    es = energy(s)
    h.step(*q, *tmp, dt, 1)
    e1 = energy(q)
    assert abs((e1 - e0) - dt * dt * es) <= 1e-5 * e0


def test_step_rejects_aliasing():
    c, f, g, h, q, tmp = _state(128, 8, 5)
    with pytest.raises(pwlib.PwError) as e:
        h.step(q[0], q[1], q[2], q[0], tmp[1], tmp[2], 1.0, 1)
    assert e.value.status == pwlib.PW_ERR_ARG


@pytest.mark.parametrize("dtype,bound", [("bf16", 0.05), ("f16", 0.01)])
def test_step_lowp_state(dtype, bound):
    """16-bit state, FP32 arithmetic, 10 steps on the smooth field with w = 0
    initially: relative error against the FP64 rollout of the original FP32
    fields stays within the stated bound (BF16 0.05, FP16 0.01 after 10 steps;
    the state is rounded once per step)."""
    nx, ny, nz = 128, 32, 16
    c0 = inputs.make_coeffs(nz)
    f = inputs.smooth_fields(nx, ny, nz, w_zero=True)
    maxabs = [max(float(x.abs().max()), 1.0) for x in f]
    sc = precision.suggest_scales(maxabs, c0, dtype)[:3]
    c, f, g, h, q, tmp = _state(nx, ny, nz, w_zero=True, dtype=dtype, scale=sc)
    h.step(*q, *tmp, 1.0, 10, scale=sc)
    h.sync()
    ref = oracle.step(*[x.numpy() for x in f], c, 1.0, 10)
    got = _dense(g, q, sc)
    for a, b in zip(got[:2], ref[:2]):
        assert np.abs(interior(a) - interior(b)).max() / np.abs(interior(b)).max() <= bound
    # w starts at 0 and grows from the u, v coupling: compare against the u scale
    assert np.abs(interior(got[2]) - interior(ref[2])).max() / np.abs(interior(ref[0])).max() <= bound


@pytest.mark.parametrize("kernel", [1, 2], ids=["generic", "tma"])
@pytest.mark.parametrize("dtype,halo,shape", [("f32", 1, (128, 24, 16)), ("f32", 2, (260, 13, 7)),
                                              ("bf16", 1, (128, 24, 16)), ("f16", 1, (132, 9, 5))])
def test_step_to_equals_one_in_place_step(kernel, dtype, halo, shape):
    """pw_step_to leaves its inputs alone and writes exactly what one step of
    pw_step leaves in place: interior and periodic halo, bit for bit."""
    nx, ny, nz = shape
    c = inputs.make_coeffs(nz)
    f = inputs.smooth_fields(nx, ny, nz, w_zero=True)
    g = pwlib.Grid(nx, ny, nz, dtype=dtype, halo=halo)
    h = pwlib.PW(g, c)
    h.set_kernel(kernel)
    sc = None
    if dtype == "f16":
        sc = precision.suggest_scales([float(x.abs().max()) for x in f], c, dtype)[:3]
    q = [g.from_dense(x, scale=s) for x, s in zip(f, sc or (1.0, 1.0, 1.0))]
    for t in q:
        h.fill_halo_periodic(t)
    before = [t.clone() for t in q]
    nxt = [g.alloc(fill=NAN) for _ in range(3)]
    h.step_to(*q, *nxt, 0.5, scale=sc)
    h.sync()
    assert h.last_kernel == kernel
    for a, b in zip(q, before):
        assert torch.equal(a.view(torch.int16) if a.element_size() == 2 else a.view(torch.int32),
                           b.view(torch.int16) if b.element_size() == 2 else b.view(torch.int32))
    tmp = [g.alloc(fill=NAN) for _ in range(3)]
    h.step(*q, *tmp, 0.5, 1, scale=sc)
    h.sync()
    for a, b in zip(nxt, q):
        assert torch.equal(g.view(a)[1:-1], g.view(b)[1:-1])
    if dtype == "f32":
        ref = oracle.step(*[x.numpy() for x in f], c, 0.5, 1)
        assert _relerr(_dense(g, nxt), ref) <= 1e-5


def test_step_to_rejections():
    nx, ny, nz = 64, 8, 5
    c, f, g, h, q, tmp = _state(nx, ny, nz)
    with pytest.raises(pwlib.PwError) as e:
        h.step_to(*q, q[0], tmp[1], tmp[2], 1.0)
    assert e.value.status == pwlib.PW_ERR_ARG
    with pytest.raises(pwlib.PwError) as e:
        h.step_to(*q, *tmp, float("nan"))
    assert e.value.status == pwlib.PW_ERR_ARG
    with pytest.raises(pwlib.PwError) as e:
        h.step_to(*q, *tmp, 1.0, scale=(1.0, 0.0, 1.0))
    assert e.value.status == pwlib.PW_ERR_ARG


def test_slab_stepper_on_one_rank_equals_pw_step():
    """The y-slab stepper (fused step kernel out of place, then the slab's
    halo exchange) on a single rank holds the whole grid, exchanges nothing,
    and gives pw_step's bits, halos included."""
    from paper_2301_13016_gb300 import slab
    nx, ny, nz, dt, n = 200, 37, 12, 1.0, 5
    c = inputs.make_coeffs(nz)
    g = pwlib.Grid(nx, ny, nz)
    h = pwlib.PW(g, c)
    f = inputs.smooth_fields(nx, ny, nz, w_zero=True)
    a = [g.from_dense(x) for x in f]
    b = [g.alloc(fill=NAN) for _ in range(3)]
    assert slab.slab_rows(ny, 1, 0) == (0, ny)
    out = slab.step_slabs(h, g, a, b, dt, n, slab.HaloExchangeY(1, 0))
    ref = [g.from_dense(x) for x in f]
    tmp = [g.alloc() for _ in range(3)]
    h.step(*ref, *tmp, dt, n)
    h.sync()
    for x, y in zip(out, ref):
        assert torch.equal(g.view(x)[1:-1], g.view(y)[1:-1])
