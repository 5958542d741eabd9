"""The CPU oracle against what the scheme and the mathematics fix (no GPU).

Tendencies: the checks in tests/pins.py (closed forms, convergence, the
discrete energy identity, symmetries, never-read levels, golden fixture).
Halo swap, time stepping and the adjoint are pinned against numpy indexing,
the energy-growth identity of forward Euler, the exact linearisation of a
quadratic map and central finite differences.
"""
import numpy as np
import pytest

import oracle
import pins
from paper_2301_13016_gb300 import inputs


def tend64(u, v, w, c):
    return oracle.tendencies(u, v, w, c, precision="f64")


def tend32(u, v, w, c):
    return tuple(a.astype(np.float64) for a in oracle.tendencies(u, v, w, c, precision="f32"))


@pytest.mark.parametrize("name", list(pins.ALL))
def test_pin_f64(name):
    err = pins.ALL[name](tend64)
    assert err <= pins.TOL[name], f"{name}: {err}"


# Single precision: the exact symmetries still hold bit for bit; the others
# hold to single-precision rounding.
F32_TOL = dict(pins.TOL, linear_exact=2e-6, energy=1e-6, energy_anelastic=1e-6, golden=1e-6)


@pytest.mark.parametrize("name", list(pins.ALL))
def test_pin_f32(name):
    err = pins.ALL[name](tend32)
    assert err <= F32_TOL[name], f"{name}: {err}"


@pytest.mark.parametrize("smooth", [False, True])
def test_f32_within_rounding_of_f64(smooth):
    nx, ny, nz = 24, 20, 10
    c = inputs.make_coeffs(nz)
    gen = inputs.smooth_fields if smooth else inputs.random_fields
    u, v, w = (f.numpy() for f in gen(nx, ny, nz))
    s64 = tend64(u, v, w, c)
    s32 = tend32(u, v, w, c)
    for a, b in zip(s64, s32):
        assert np.abs(a - b).max() / np.abs(a).max() < 1e-5


def test_outputs_halo_untouched_and_lid_zero():
    nx, ny, nz = 8, 6, 5
    c = inputs.make_coeffs(nz)
    u, v, w = (f.numpy() for f in inputs.random_fields(nx, ny, nz))
    su, sv, sw = tend64(u, v, w, c)
    for s in (su, sv, sw):
        assert np.all(s[0] == 0) and np.all(s[nz + 1] == 0)
        assert np.all(s[:, 0] == 0) and np.all(s[:, ny + 1] == 0)
        assert np.all(s[:, :, 0] == 0) and np.all(s[:, :, nx + 1] == 0)
        assert np.all(s[1] == 0)
    assert np.all(sw[nz] == 0)
    assert np.abs(su[nz]).max() > 0 and np.abs(sv[nz]).max() > 0


def test_fill_halo_matches_wrap_padding():
    rng = np.random.default_rng(3)
    nx, ny, nz = 7, 5, 4
    f = rng.normal(size=(nz + 2, ny + 2, nx + 2))
    g = oracle.fill_halo_periodic(f)
    ref = np.pad(f[1:-1, 1:-1, 1:-1], ((0, 0), (1, 1), (1, 1)), mode="wrap")
    assert np.array_equal(g[1:-1], ref)
    assert np.array_equal(g[0], f[0]) and np.array_equal(g[nz + 1], f[nz + 1])


def _interior(f):
    return f[1:-1, 1:-1, 1:-1]


def test_step_energy_growth_identity():
    """With the discrete energy identity sum W q.s = 0, one Euler step gives
    ||q + dt s||_W^2 = ||q||_W^2 + dt^2 ||s||_W^2 exactly (up to rounding)."""
    nx, ny, nz = 8, 6, 7
    c = inputs.make_coeffs(nz, anelastic=True)
    u, v, w = (f.numpy().astype(np.float64) for f in inputs.random_fields(nx, ny, nz))
    dt = 0.37
    s = tend64(u, v, w, c)
    u1, v1, w1 = oracle.step(u, v, w, c, dt, 1)
    wu = (c.rho_u * c.dz_u)[:, None, None]
    ww = (c.rho_w * c.dz_w)[:, None, None]

    def norm(q, wt, lo, hi):
        return float(np.sum(wt[lo:hi + 1] * q[lo:hi + 1, 1:-1, 1:-1] ** 2))

    for q0, q1, sq, wt, lo, hi in ((u, u1, s[0], wu, 2, nz), (v, v1, s[1], wu, 2, nz),
                                  (w, w1, s[2], ww, 2, nz - 1)):
        lhs = norm(q1, wt, lo, hi)
        rhs = norm(q0, wt, lo, hi) + dt * dt * norm(sq, wt, lo, hi)
        assert abs(lhs - rhs) / rhs < 1e-13


def test_step_composes_and_refills_halo():
    nx, ny, nz = 6, 5, 5
    c = inputs.make_coeffs(nz)
    u, v, w = (f.numpy().astype(np.float64) for f in inputs.random_fields(nx, ny, nz))
    a = oracle.step(u, v, w, c, 0.5, 2)
    b = oracle.step(*oracle.step(u, v, w, c, 0.5, 1), c, 0.5, 1)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
        assert np.array_equal(x, oracle.fill_halo_periodic(x))
    # surface and lid values of w, surface values of u and v do not move
    assert np.array_equal(a[2][1], w[1]) and np.array_equal(a[2][nz], w[nz])
    assert np.array_equal(_interior(a[0])[0], _interior(u)[0])


def _rand(shape, seed):
    return np.random.default_rng(seed).normal(size=shape)


@pytest.mark.parametrize("anelastic", [False, True])
def test_adjoint_dot_product(anelastic):
    """<l, J(q) d> = <J(q)^T l, d>, with J(q) d = s(q+d) - s(q) - s(d) exact
    for the quadratic map s (so the check rests on the pinned tendencies)."""
    nx, ny, nz = 6, 5, 6
    c = inputs.make_coeffs(nz, anelastic=anelastic)
    shape = (nz + 2, ny + 2, nx + 2)
    q = [_rand(shape, 1), _rand(shape, 2), _rand(shape, 3)]
    d = [_rand(shape, 4), _rand(shape, 5), _rand(shape, 6)]
    lam = [_rand(shape, 7), _rand(shape, 8), _rand(shape, 9)]
    s_qd = tend64(*[a + b for a, b in zip(q, d)], c)
    s_q = tend64(*q, c)
    s_d = tend64(*d, c)
    jd = [a - b - e for a, b, e in zip(s_qd, s_q, s_d)]
    lhs = sum(float(np.sum(l * x)) for l, x in zip(lam, jd))
    g = oracle.adjoint_tendencies(*q, c, *lam)
    rhs = sum(float(np.sum(x * y)) for x, y in zip(g, d))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)
    # J(q) q = 2 s(q)
    lhs2 = sum(float(np.sum(l * 2 * x)) for l, x in zip(lam, s_q))
    rhs2 = sum(float(np.sum(x * y)) for x, y in zip(g, q))
    assert abs(lhs2 - rhs2) <= 1e-12 * max(abs(lhs2), 1.0)


def test_fold_is_transpose_of_fill():
    nx, ny, nz = 5, 4, 3
    shape = (nz + 2, ny + 2, nx + 2)
    f = _rand(shape, 1)
    f[0] = 0
    f[nz + 1] = 0
    g = _rand(shape, 2)
    g[0] = 0
    g[nz + 1] = 0
    fi = np.zeros(shape)
    fi[1:-1, 1:-1, 1:-1] = f[1:-1, 1:-1, 1:-1]
    lhs = float(np.sum(g * oracle.fill_halo_periodic(fi)))
    rhs = float(np.sum(oracle.fold_halo_periodic(g) * fi))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_step_adjoint_matches_central_differences():
    """dL/de of L = 1/2 sum (u_T - u_t)^2 along a direction d, by central
    differences of the float64 rollout, against <g_0, d> from the reverse sweep."""
    nx, ny, nz = 6, 5, 6
    c = inputs.make_coeffs(nz)
    u, v, w = (f.numpy().astype(np.float64) for f in inputs.smooth_fields(nx, ny, nz))
    w = w * 0.5
    w[1] = 0
    w[nz] = 0
    dt, nsteps = 0.5, 4
    shape = u.shape
    ut = _rand(shape, 5)
    d = [_rand(shape, 6), _rand(shape, 7), _rand(shape, 8)]
    for x in d:
        x[0] = x[nz + 1] = 0
        x[:, 0] = x[:, -1] = 0
        x[:, :, 0] = x[:, :, -1] = 0
    d[2][1] = d[2][nz] = 0

    def loss(a, b, e):
        uT, _, _ = oracle.step(a, b, e, c, dt, nsteps)
        return 0.5 * float(np.sum((_interior(uT) - _interior(ut)) ** 2))

    uT, vT, wT = oracle.step(u, v, w, c, dt, nsteps)
    gu = np.zeros(shape)
    gu[1:-1, 1:-1, 1:-1] = _interior(uT) - _interior(ut)
    g = oracle.step_adjoint(u, v, w, c, dt, nsteps, gu, np.zeros(shape), np.zeros(shape))
    ana = sum(float(np.sum(x * y)) for x, y in zip(g, d))
    eps = 1e-4
    fd = (loss(u + eps * d[0], v + eps * d[1], w + eps * d[2])
          - loss(u - eps * d[0], v - eps * d[1], w - eps * d[2])) / (2 * eps)
    assert abs(fd - ana) <= 1e-7 * abs(ana)


def test_abs_terms_bounds_and_pins():
    nx, ny, nz = 8, 6, 7
    c = inputs.make_coeffs(nz, anelastic=True)
    u, v, w = (f.numpy().astype(np.float64) for f in inputs.random_fields(nx, ny, nz))
    s = tend64(u, v, w, c)
    a = oracle.abs_terms(u, v, w, c)
    for si, ai in zip(s, a):
        assert np.all(ai >= np.abs(si) * (1 - 1e-15))        # triangle inequality
    a2 = oracle.abs_terms(2 * u, 2 * v, 2 * w, c)
    for x, y in zip(a, a2):
        assert np.array_equal(4 * x, y)
    # single nonzero term: u only at (k,j,i-1) and (k,j,i) -> su(k,j,i) has the
    # one x-term tcx*u(i-1)*(u+u(i-1)) with b, d of one sign: equality
    z = np.zeros_like(u)
    uu = z.copy()
    uu[3, 3, 3] = 1.5
    uu[3, 3, 4] = 0.5
    s1 = tend64(uu, z, z, c)
    a1 = oracle.abs_terms(uu, z, z, c)
    assert s1[0][3, 3, 4] != 0 and a1[0][3, 3, 4] == abs(s1[0][3, 3, 4])
    # the FP32 oracle's rounding error sits inside a small multiple of u32 * sum
    s32 = tend32(u, v, w, c)
    for x, y, ai in zip(s32, s, a):
        assert np.all(np.abs(x - y) <= 16 * 2.0 ** -24 * ai + 1e-300)


def _scatter_face_by_face(u, v, w, c):
    """The scheme restated face by face, the way a flux-form code scatters:
    across each face between cells A and B = A + e, with advecting pair sum P
    on that face, cell B receives +coef * phi(A) * P and cell A receives
    -coef' * phi(B) * P (Sec. 2.2's terms c * a * (b + d), grouped by face
    instead of by output cell).  Only cells where the scheme has outputs
    receive: su, sv at levels 2..nz (the upper vertical term up to nz-1), sw
    at 2..nz-1, interior columns.  An index cross-check of the oracle's
    gather loops (the same terms, in a different arrangement), not an
    independent pin."""
    nz, ny, nx = u.shape[0] - 2, u.shape[1] - 2, u.shape[2] - 2
    su, sv, sw = np.zeros(u.shape), np.zeros(u.shape), np.zeros(u.shape)
    inside = lambda j, i: 1 <= j <= ny and 1 <= i <= nx

    def face(s, phi, coef_b, coef_a, P, A, B, ok_a, ok_b):
        if ok_b and inside(*B[1:]):
            s[B] += coef_b * phi[A] * P
        if ok_a and inside(*A[1:]):
            s[A] -= coef_a * phi[B] * P

    for k in range(1, nz + 1):
        uv_k = 2 <= k <= nz
        w_k = 2 <= k <= nz - 1
        for j in range(0, ny + 2):
            for i in range(1, nx + 2):           # x faces between i-1 and i
                A, B = (k, j, i - 1), (k, j, i)
                face(su, u, c.tcx, c.tcx, u[k, j, i - 1] + u[k, j, i], A, B, uv_k, uv_k)
                if j <= ny:
                    face(sv, v, c.tcx, c.tcx, u[k, j, i - 1] + u[k, j + 1, i - 1], A, B, uv_k, uv_k)
                if k <= nz - 1:
                    face(sw, w, c.tcx, c.tcx, u[k, j, i - 1] + u[k + 1, j, i - 1], A, B, w_k, w_k)
        for j in range(1, ny + 2):               # y faces between j-1 and j
            for i in range(0, nx + 2):
                A, B = (k, j - 1, i), (k, j, i)
                if i <= nx:
                    face(su, u, c.tcy, c.tcy, v[k, j - 1, i] + v[k, j - 1, i + 1], A, B, uv_k, uv_k)
                face(sv, v, c.tcy, c.tcy, v[k, j - 1, i] + v[k, j, i], A, B, uv_k, uv_k)
                if k <= nz - 1:
                    face(sw, w, c.tcy, c.tcy, v[k, j - 1, i] + v[k + 1, j - 1, i], A, B, w_k, w_k)
    for k in range(2, nz + 1):                   # z faces between k-1 and k
        for j in range(0, ny + 2):
            for i in range(0, nx + 2):
                A, B = (k - 1, j, i), (k, j, i)
                up_ok = 2 <= k - 1 <= nz - 1     # the upper vertical term of level k-1
                if i <= nx:
                    face(su, u, c.tzc1[k], c.tzc2[k - 1], w[k - 1, j, i] + w[k - 1, j, i + 1], A, B, up_ok, True)
                if j <= ny:
                    face(sv, v, c.tzc1[k], c.tzc2[k - 1], w[k - 1, j, i] + w[k - 1, j + 1, i], A, B, up_ok, True)
                face(sw, w, c.tzd1[k], c.tzd2[k - 1], w[k - 1, j, i] + w[k, j, i], A, B, up_ok, k <= nz - 1)
    return su, sv, sw


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_face_by_face_scatter_on_4cubed_dyadic_grids(seed):
    """4 x 4 x 4 interior with dyadic values (multiples of 1/4 in -2..2) and
    dyadic coefficients (multiples of 1/8): every product and sum is exact in
    FP64, so the scatter restatement and the oracle agree bit for bit."""
    rng = np.random.default_rng(seed)
    n = 4
    shape = (n + 2, n + 2, n + 2)
    u, v, w = (rng.integers(-8, 9, size=shape) / 4.0 for _ in range(3))
    c = inputs.make_coeffs(n)
    c.tcx, c.tcy = 0.25, 0.5
    for name in ("tzc1", "tzc2", "tzd1", "tzd2"):
        setattr(c, name, rng.integers(1, 9, size=n + 2) / 8.0)
    ref = _scatter_face_by_face(u, v, w, c)
    got = tend64(u, v, w, c)
    for g, r in zip(got, ref):
        assert np.array_equal(g[1:-1, 1:-1, 1:-1], r[1:-1, 1:-1, 1:-1])
        assert np.any(r[1:-1, 1:-1, 1:-1] != 0)
