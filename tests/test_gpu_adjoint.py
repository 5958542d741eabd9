"""pw_adjoint and the autograd rollout through the C ABI, against the oracle.

  * full-array adjoint vs oracle.adjoint_tendencies on every cell it writes;
  * periodic adjoint vs the oracle's adjoint folded onto the interior, for
    the generic kernel and every instantiated TMA launch shape;
  * ACCUMULATE and ADD_LAMBDA modes;
  * the rollout gradient (PWRollout, checkpointed) vs oracle.step_adjoint and
    vs central finite differences of the GPU rollout.
Bar: max|err| / max|ref| <= 1e-5 (FP32 arithmetic against FP64) for single
evaluations, 1e-4 for multi-step reverse sweeps.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2301_13016_gb300 as pwlib
from paper_2301_13016_gb300 import inputs
from paper_2301_13016_gb300.autograd import rollout
from gpu_util import NAN

pytestmark = pytest.mark.gpu


def _rand_dense(nx, ny, nz, seed):
    g = torch.Generator().manual_seed(seed)
    return torch.randn((nz + 2, ny + 2, nx + 2), generator=g, dtype=torch.float32)


def _setup(nx, ny, nz, anelastic=False, periodic_q=False):
    c = inputs.make_coeffs(nz, anelastic=anelastic)
    q = [_rand_dense(nx, ny, nz, s) * 5 for s in (1, 2, 3)]
    if periodic_q:
        for x in q:
            inputs.wrap_halo_(x)
    lam = [_rand_dense(nx, ny, nz, s) for s in (4, 5, 6)]
    g = pwlib.Grid(nx, ny, nz)
    h = pwlib.PW(g, c)
    dq = [g.from_dense(x) for x in q]
    dl = [g.from_dense(x) for x in lam]
    return c, q, lam, g, h, dq, dl


def _written_region(g):
    """levels 1..nz, interior plus one-cell lateral halo"""
    return (slice(1, g.nz + 1), slice(0, g.ny + 2), slice(0, g.nx + 2))


@pytest.mark.parametrize("shape", [(64, 12, 8), (37, 9, 5), (5, 4, 3)])
@pytest.mark.parametrize("anelastic", [False, True])
def test_adjoint_full_array_matches_oracle(shape, anelastic):
    c, q, lam, g, h, dq, dl = _setup(*shape, anelastic=anelastic)
    out = [g.alloc(fill=NAN) for _ in range(3)]
    h.adjoint(*dq, *dl, *out, alpha=1.0, flags=0)
    h.sync()
    ref = oracle.adjoint_tendencies(*[x.numpy() for x in q], c, *[x.numpy() for x in lam])
    reg = _written_region(g)
    for o, r in zip(out, ref):
        got = g.to_dense(o).numpy()[reg]
        rr = r[reg]
        assert np.all(np.isfinite(got))
        assert np.abs(got - rr).max() <= 1e-5 * np.abs(rr).max()
        # the z-halo planes are not written
        v = g.view(o)
        assert torch.isnan(v[0]).all() and torch.isnan(v[-1]).all()


@pytest.mark.parametrize("shape", [(64, 12, 8), (36, 7, 6), (260, 9, 5), (128, 16, 20)])
@pytest.mark.parametrize("kernel", [1, 2], ids=["generic", "tma"])
@pytest.mark.parametrize("anelastic", [False, True], ids=["boussinesq", "anelastic"])
def test_adjoint_periodic_matches_folded_oracle(shape, kernel, anelastic):
    c, q, lam, g, h, dq, dl = _setup(*shape, anelastic=anelastic, periodic_q=True)
    out = [g.alloc(fill=NAN) for _ in range(3)]
    h.set_kernel(kernel)
    h.adjoint(*dq, *dl, *out, alpha=1.0, flags=pwlib.PW_ADJ_PERIODIC)
    h.sync()
    assert h.last_kernel == kernel
    # the oracle's adjoint sees the lambda entries at the scheme's outputs only
    lam_int = []
    for x in lam:
        y = np.zeros(x.shape)
        y[1:-1, 1:-1, 1:-1] = x.numpy()[1:-1, 1:-1, 1:-1]
        lam_int.append(y)
    full = oracle.adjoint_tendencies(*[x.numpy() for x in q], c, *lam_int)
    for o, r in zip(out, full):
        ref = oracle.fold_halo_periodic(r)[1:-1, 1:-1, 1:-1]
        got = g.to_dense(o).numpy()[1:-1, 1:-1, 1:-1]
        assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
        v = g.view(o)
        assert torch.isnan(v[1:-1, 0]).all() and torch.isnan(v[1:-1, :, 0]).all()   # halo not written


ADJ_SHAPES = [(4, 5, 4), (4, 4, 4), (4, 6, 4), (2, 4, 4), (2, 5, 4), (2, 6, 4), (2, 8, 4), (2, 8, 3)]


@pytest.mark.parametrize("cfg", ADJ_SHAPES, ids=[f"c{a}_ty{b}_s{c}" for a, b, c in ADJ_SHAPES])
def test_adjoint_tma_shapes_match_folded_oracle(cfg):
    """Every instantiated TMA adjoint shape on a grid ragged in x (260 = 2 x 128
    + 4 = 4 x 64 + 4), in y (19 rows) and in z (4 k segments of 10 levels)."""
    c, q, lam, g, h, dq, dl = _setup(260, 19, 40, periodic_q=True)
    h.set_adjoint_config(*cfg, nseg=4)
    assert h.adjoint_config() == dict(zip(("cells", "ty", "stages", "nseg"), cfg + (4,)))
    out = [g.alloc(fill=NAN) for _ in range(3)]
    h.adjoint(*dq, *dl, *out, alpha=1.0, flags=pwlib.PW_ADJ_PERIODIC)
    h.sync()
    assert h.last_kernel == 2
    lam_int = []
    for x in lam:
        y = np.zeros(x.shape)
        y[1:-1, 1:-1, 1:-1] = x.numpy()[1:-1, 1:-1, 1:-1]
        lam_int.append(y)
    full = oracle.adjoint_tendencies(*[x.numpy() for x in q], c, *lam_int)
    for o, r in zip(out, full):
        ref = oracle.fold_halo_periodic(r)[1:-1, 1:-1, 1:-1]
        got = g.to_dense(o).numpy()[1:-1, 1:-1, 1:-1]
        assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
        v = g.view(o)
        assert torch.isnan(v[1:-1, 0]).all() and torch.isnan(v[1:-1, :, 0]).all()   # halo not written


def test_adjoint_config_rejections():
    g = pwlib.Grid(64, 8, 4)
    h = pwlib.PW(g, inputs.make_coeffs(4))
    auto = h.adjoint_config()
    assert (auto["cells"], auto["ty"], auto["stages"]) in ADJ_SHAPES and auto["nseg"] == 1
    for bad in [(3, 0, 0), (2, 7, 4), (4, 8, 4)]:
        with pytest.raises(pwlib.PwError) as e:
            h.set_adjoint_config(*bad)
        assert e.value.status == pwlib.PW_ERR_UNSUPPORTED
    for bad in [(-1, 0, 0, 0), (0, 0, 0, 5), (0, 0, 0, -1)]:
        with pytest.raises(pwlib.PwError) as e:
            h.set_adjoint_config(*bad)
        assert e.value.status == pwlib.PW_ERR_ARG
    assert h.adjoint_config() == auto


@pytest.mark.parametrize("kernel", [1, 2], ids=["generic", "tma"])
def test_adjoint_accumulate_and_add_lambda(kernel):
    c, q, lam, g, h, dq, dl = _setup(64, 10, 6, periodic_q=True)
    h.set_kernel(kernel)
    base = [g.from_dense(_rand_dense(64, 10, 6, s)) for s in (7, 8, 9)]
    plain = [g.alloc() for _ in range(3)]
    h.adjoint(*dq, *dl, *plain, alpha=0.5, flags=pwlib.PW_ADJ_PERIODIC)
    acc = [b.clone() for b in base]
    h.adjoint(*dq, *dl, *acc, alpha=0.5, flags=pwlib.PW_ADJ_PERIODIC | pwlib.PW_ADJ_ACCUMULATE)
    addl = [g.alloc() for _ in range(3)]
    h.adjoint(*dq, *dl, *addl, alpha=0.5, flags=pwlib.PW_ADJ_PERIODIC | pwlib.PW_ADJ_ADD_LAMBDA)
    h.sync()
    for p_, a_, b_, l_, x_ in zip(plain, acc, base, dl, addl):
        vi = lambda t: g.view(t)[1:-1, 1:-1, 1:-1]
        assert torch.allclose(vi(a_), vi(b_) + vi(p_), rtol=1e-6, atol=1e-6)
        assert torch.allclose(vi(x_), vi(l_) + vi(p_), rtol=1e-6, atol=1e-6)
    with pytest.raises(pwlib.PwError):
        h.adjoint(*dq, *dl, *acc, flags=pwlib.PW_ADJ_ACCUMULATE | pwlib.PW_ADJ_ADD_LAMBDA)
    with pytest.raises(pwlib.PwError):
        h.adjoint(*dq, *dl, dl[0], acc[1], acc[2])


def test_adjoint_rejects_16bit_storage():
    g = pwlib.Grid(64, 8, 4, dtype="bf16")
    h = pwlib.PW(g, inputs.make_coeffs(4))
    t = [g.alloc() for _ in range(9)]
    with pytest.raises(pwlib.PwError) as e:
        h.adjoint(*t)
    assert e.value.status == pwlib.PW_ERR_UNSUPPORTED


def _rollout_case(nx, ny, nz, nsteps, every, dt=1.0):
    c = inputs.make_coeffs(nz)
    f = inputs.smooth_fields(nx, ny, nz, w_zero=True)
    g = pwlib.Grid(nx, ny, nz)
    h = pwlib.PW(g, c)
    q0 = [g.from_dense(x).requires_grad_(True) for x in f]
    ut = inputs.target_field(nx, ny, nz)
    return c, f, g, h, q0, ut


def _loss(g, uT, ut):
    d = g.view(uT)[1:-1, 1:-1, 1:-1].double() - ut[1:-1, 1:-1, 1:-1].to(uT.device).double()
    return 0.5 * (d * d).sum()


@pytest.mark.parametrize("nsteps,every", [(6, 2), (7, 5), (4, 10)])
def test_rollout_gradient_matches_oracle(nsteps, every):
    nx, ny, nz = 64, 24, 16
    dt = 1.0
    c, f, g, h, q0, ut = _rollout_case(nx, ny, nz, nsteps, every, dt)
    uT, vT, wT = rollout(*q0, h, dt, nsteps, every)
    L = _loss(g, uT, ut)
    L.backward()
    # oracle: forward in FP64 from the same FP32 start, reverse sweep in FP64
    qT = oracle.step(*[x.numpy() for x in f], c, dt, nsteps)
    gT = np.zeros(qT[0].shape)
    gT[1:-1, 1:-1, 1:-1] = qT[0][1:-1, 1:-1, 1:-1] - ut.numpy()[1:-1, 1:-1, 1:-1]
    ref = oracle.step_adjoint(*[x.numpy() for x in f], c, dt, nsteps, gT, np.zeros_like(gT), np.zeros_like(gT))
    for t, r in zip(q0, ref):
        got = g.to_dense(t.grad).numpy()
        assert np.abs(got[1:-1, 1:-1, 1:-1] - r[1:-1, 1:-1, 1:-1]).max() <= 1e-4 * np.abs(r).max()
        assert np.all(got[:, 0] == 0) and np.all(got[:, :, 0] == 0)     # halo entries carry no gradient


def test_rollout_gradient_central_differences():
    """dL/de along a direction supported on an 8^3 sub-box: central differences
    of the GPU rollout (loss summed in FP64) against <grad, d>."""
    nx, ny, nz = 64, 24, 16
    nsteps, every, dt = 6, 3, 1.0
    c, f, g, h, q0, ut = _rollout_case(nx, ny, nz, nsteps, every, dt)
    uT, vT, wT = rollout(*q0, h, dt, nsteps, every)
    L = _loss(g, uT, ut)
    L.backward()
    gen = torch.Generator().manual_seed(99)
    d = []
    for n in range(3):
        x = torch.zeros((nz + 2, ny + 2, nx + 2))
        x[5:13, 8:16, 20:28] = torch.randn((8, 8, 8), generator=gen)
        if n == 2:
            x[1] = 0
            x[nz] = 0
        d.append(x)
    dd = [g.from_dense(x) for x in d]
    ana = sum(float((t.grad.double() * e.double()).sum()) for t, e in zip(q0, dd))
    eps = 1e-2

    def L_at(s):
        with torch.no_grad():
            q = [(t.detach() + s * e) for t, e in zip(q0, dd)]
            out = rollout(*q, h, dt, nsteps, every)
            return float(_loss(g, out[0], ut))

    fd = (L_at(eps) - L_at(-eps)) / (2 * eps)
    assert abs(fd - ana) <= 2e-3 * abs(ana)


def test_rollout_forward_equals_in_place_steps():
    """The rollout's out-of-place steps give the bits of pw_step run in place,
    and the returned state holds no unset entries."""
    nx, ny, nz = 64, 24, 16
    c, f, g, h, q0, ut = _rollout_case(nx, ny, nz, 7, 3)
    outs = rollout(*q0, h, 1.0, 7, 3)
    q = [t.detach().clone() for t in q0]
    tmp = [g.alloc() for _ in range(3)]
    h.step(*q, *tmp, 1.0, 7)
    h.sync()
    for a, b in zip(outs, q):
        assert torch.equal(g.view(a)[1:-1], g.view(b)[1:-1])
        assert torch.isfinite(a).all()
    z = rollout(*q0, h, 1.0, 0, 3)
    for a, b in zip(z, q0):
        assert torch.equal(g.view(a)[1:-1, 1:-1, 1:-1], g.view(b)[1:-1, 1:-1, 1:-1].detach())
