"""Checks that pin the oracle's tendencies to facts outside the oracle itself.

Each check takes `tend(u, v, w, coeffs) -> (su, sv, sw)` (numpy float64, dense
(nz+2, ny+2, nx+2) layout) and returns a non-negative error figure; the caller
compares it with the check's threshold (TOL).  The same checks run on the
real oracle (tests/test_oracle_pins.py) and on deliberately broken copies of
it (tests/test_oracle_mutants.py), which must each fail at least one check.

What the checks use:
  * the continuous operator the scheme discretises: the skew-symmetric
    momentum advection  S(q) = -1/2 [ (u.grad) q + div(u q) ]
                              = -(u.grad) q - 1/2 q div(u);
    on a uniform grid the discrete scheme reproduces it exactly for fields
    linear in x, y, z, and to second order for smooth fields;
  * the discrete kinetic-energy identity that defines the PW scheme's
    conservation property: with periodic x, y and w = 0 on surface and lid,
    sum_k W_k sum_ij q s = 0 for q = u, v (weights rho_u dz_u) and q = w
    (weights rho_w dz_w), for arbitrary fields;
  * exact symmetries: mirror antisymmetry in x and y, quadratic scaling;
  * levels the scheme never reads (z-halo planes) filled with NaN.
"""
import json
import math
import os

import numpy as np

from paper_2301_13016_gb300 import inputs

TOL = {
    "uniform_zero": 0.0,
    "linear_exact": 1e-12,
    "convergence": 0.25,     # |observed order - 2|
    "energy": 1e-12,
    "energy_anelastic": 1e-12,
    "mirror_x": 0.0,
    "mirror_y": 0.0,
    "quadratic": 0.0,
    "zhalo": 0.0,
    "golden": 1e-12,
}

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _zeros(nx, ny, nz):
    return np.zeros((nz + 2, ny + 2, nx + 2))


def _wrap(f):
    return inputs.wrap_halo_(f)


def _rand_periodic(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    out = []
    for n in range(3):
        f = _zeros(nx, ny, nz)
        f[1:-1, 1:-1, 1:-1] = rng.normal(size=(nz, ny, nx))
        if n == 2:
            f[1] = 0.0
            f[nz] = 0.0
        _wrap(f)
        out.append(f)
    return out


# ---------------------------------------------------------------------------
# staggered positions of the Arakawa-C grid: u(k,j,i) at (i dx, (j-1/2) dy, z_u[k]),
# v at ((i-1/2) dx, j dy, z_u[k]), w at ((i-1/2) dx, (j-1/2) dy, z_w[k]).
def _positions(nx, ny, nz, dx, dy, c):
    K, J, I = np.meshgrid(np.arange(nz + 2), np.arange(ny + 2), np.arange(nx + 2), indexing="ij")
    zu = c.z_u[K]
    zw = c.z_w[K]
    pu = (I * dx, (J - 0.5) * dy, zu)
    pv = ((I - 0.5) * dx, J * dy, zu)
    pw = ((I - 0.5) * dx, (J - 0.5) * dy, zw)
    return pu, pv, pw


def continuous_S(vel, grad, q_index, pos):
    """-(u.grad) q - 1/2 q div(u) at `pos`, from callables vel[b](x,y,z) and
    grad[a][b](x,y,z) = d vel[a] / d x_b."""
    x, y, z = pos
    vals = [vel[b](x, y, z) for b in range(3)]
    adv = sum(vals[b] * grad[q_index][b](x, y, z) for b in range(3))
    div = sum(grad[b][b](x, y, z) for b in range(3))
    return -adv - 0.5 * vals[q_index] * div


def pin_uniform_zero(tend):
    nx, ny, nz = 6, 5, 6
    c = inputs.make_coeffs(nz)
    u = _zeros(nx, ny, nz) + 3.25
    v = _zeros(nx, ny, nz) - 1.5
    w = _zeros(nx, ny, nz)
    s = tend(u, v, w, c)
    return float(max(np.abs(a).max() for a in s))


def _linear_case(nx, ny, nz, dx, dy, dz, A):
    c = inputs.make_coeffs(nz, dx=dx, dy=dy, uniform_dz=dz)
    pu, pv, pw = _positions(nx, ny, nz, dx, dy, c)
    lin = [lambda x, y, z, a=A[n]: a[0] + a[1] * x + a[2] * y + a[3] * z for n in range(3)]
    grad = [[(lambda x, y, z, g=A[n][1 + b]: g + 0 * x) for b in range(3)] for n in range(3)]
    u = lin[0](*pu)
    v = lin[1](*pv)
    w = lin[2](*pw)
    return c, (u, v, w), (pu, pv, pw), lin, grad


def pin_linear_exact(tend):
    """Fields linear in x, y, z on a uniform grid: the scheme equals the
    continuous operator exactly at every level 2..nz-1 (the lid level drops its
    upper flux by construction).  dx != dy so tcx and tcy cannot be swapped."""
    nx, ny, nz = 5, 4, 6
    dx, dy, dz = 100.0, 80.0, 50.0
    A = np.array([[1.0, 2.0, -1.0, 3.0], [-2.0, 1.0, 2.0, -1.0], [0.5, -3.0, 1.0, 2.0]]) * 1e-2
    A[:, 0] *= 100.0
    c, (u, v, w), pos, lin, grad = _linear_case(nx, ny, nz, dx, dy, dz, A)
    su, sv, sw = tend(u, v, w, c)
    err, ref = 0.0, 0.0
    for q, (s, p) in enumerate(zip((su, sv, sw), pos)):
        exact = continuous_S(lin, grad, q, p)
        sl = (slice(2, nz), slice(1, ny + 1), slice(1, nx + 1))
        err = max(err, float(np.abs(s[sl] - exact[sl]).max()))
        ref = max(ref, float(np.abs(exact[sl]).max()))
    return err / ref


def pin_convergence(tend):
    """Smooth non-polynomial fields on uniform grids of spacing h and h/2: the
    error against the continuous operator falls by about 4 (second order; the
    observed order on 16^3 -> 32^3 is 1.87-2.0).  Returns
    |observed order - 2| (worst over the three fields)."""
    L = 1000.0
    kx, ky, kz = 2 * np.pi / L * np.array([1.0, 2.0, 1.5])
    vel = [
        lambda x, y, z: 3 + np.sin(kx * x + 0.3) * np.cos(ky * y) + 0.5 * np.sin(kz * z),
        lambda x, y, z: -1 + np.cos(kx * x) * np.sin(ky * y + 0.7) + 0.3 * np.cos(kz * z),
        lambda x, y, z: 2 + np.sin(kx * x + ky * y) * np.cos(kz * z + 0.2),
    ]
    grad = [
        [lambda x, y, z: kx * np.cos(kx * x + 0.3) * np.cos(ky * y),
         lambda x, y, z: -ky * np.sin(kx * x + 0.3) * np.sin(ky * y),
         lambda x, y, z: 0.5 * kz * np.cos(kz * z)],
        [lambda x, y, z: -kx * np.sin(kx * x) * np.sin(ky * y + 0.7),
         lambda x, y, z: ky * np.cos(kx * x) * np.cos(ky * y + 0.7),
         lambda x, y, z: -0.3 * kz * np.sin(kz * z)],
        [lambda x, y, z: kx * np.cos(kx * x + ky * y) * np.cos(kz * z + 0.2),
         lambda x, y, z: ky * np.cos(kx * x + ky * y) * np.cos(kz * z + 0.2),
         lambda x, y, z: -kz * np.sin(kx * x + ky * y) * np.sin(kz * z + 0.2)],
    ]
    errs = []
    for n in (16, 32):
        h = L / n
        nx = ny = nz = n
        c = inputs.make_coeffs(nz, dx=h, dy=h, uniform_dz=h)
        pos = _positions(nx, ny, nz, h, h, c)
        fields = [vel[q](*pos[q]) for q in range(3)]
        s = tend(*fields, c)
        e = []
        for q in range(3):
            exact = continuous_S(vel, grad, q, pos[q])
            sl = (slice(2, nz), slice(1, ny + 1), slice(1, nx + 1))
            e.append(float(np.abs(s[q][sl] - exact[sl]).max()))
        errs.append(e)
    order = [math.log2(errs[0][q] / errs[1][q]) if errs[1][q] > 0 else 0.0 for q in range(3)]
    return max(abs(o - 2.0) for o in order)


def _energy(tend, anelastic):
    nx, ny, nz = 6, 5, 7
    c = inputs.make_coeffs(nz, dx=100.0, dy=90.0, anelastic=anelastic)
    u, v, w = _rand_periodic(nx, ny, nz, seed=7)
    su, sv, sw = tend(u, v, w, c)
    I = slice(1, nx + 1)
    J = slice(1, ny + 1)
    worst = 0.0
    for q, s, lo, hi, wt in ((u, su, 2, nz, c.rho_u * c.dz_u), (v, sv, 2, nz, c.rho_u * c.dz_u),
                             (w, sw, 2, nz - 1, c.rho_w * c.dz_w)):
        terms = np.array([wt[k] * np.sum(q[k, J, I] * s[k, J, I]) for k in range(lo, hi + 1)])
        scale = sum(wt[k] * np.sum(np.abs(q[k, J, I] * s[k, J, I])) for k in range(lo, hi + 1))
        worst = max(worst, abs(terms.sum()) / scale)
    return worst


def pin_energy(tend):
    return _energy(tend, anelastic=False)


def pin_energy_anelastic(tend):
    return _energy(tend, anelastic=True)


def pin_mirror_x(tend):
    """x -> -x: u'(i) = -u(N-i) (periodic index), v'(i) = v(N+1-i), w'(i) = w(N+1-i)
    gives su'(i) = -su(N-i), sv'(i) = sv(N+1-i), sw'(i) = sw(N+1-i), bit for bit."""
    nx, ny, nz = 6, 5, 6
    c = inputs.make_coeffs(nz)
    u, v, w = _rand_periodic(nx, ny, nz, seed=11)
    N = nx
    iu = np.array([(N - i - 1) % N + 1 for i in range(1, N + 1)])    # N-i, periodic in 1..N
    ic = np.array([N + 1 - i for i in range(1, N + 1)])
    up, vp, wp = (_zeros(nx, ny, nz) for _ in range(3))
    up[1:-1, 1:-1, 1:-1] = -u[1:-1, 1:-1, iu]
    vp[1:-1, 1:-1, 1:-1] = v[1:-1, 1:-1, ic]
    wp[1:-1, 1:-1, 1:-1] = w[1:-1, 1:-1, ic]
    for f in (up, vp, wp):
        _wrap(f)
    su, sv, sw = tend(u, v, w, c)
    sup, svp, swp = tend(up, vp, wp, c)
    d = max(np.abs(sup[1:-1, 1:-1, 1:-1] + su[1:-1, 1:-1, iu]).max(),
            np.abs(svp[1:-1, 1:-1, 1:-1] - sv[1:-1, 1:-1, ic]).max(),
            np.abs(swp[1:-1, 1:-1, 1:-1] - sw[1:-1, 1:-1, ic]).max())
    return float(d)


def pin_mirror_y(tend):
    """y -> -y: v'(j) = -v(N-j) (periodic index), u'(j) = u(N+1-j), w'(j) = w(N+1-j)."""
    nx, ny, nz = 5, 6, 6
    c = inputs.make_coeffs(nz)
    u, v, w = _rand_periodic(nx, ny, nz, seed=13)
    N = ny
    jv = np.array([(N - j - 1) % N + 1 for j in range(1, N + 1)])
    jc = np.array([N + 1 - j for j in range(1, N + 1)])
    up, vp, wp = (_zeros(nx, ny, nz) for _ in range(3))
    vp[1:-1, 1:-1, 1:-1] = -v[1:-1, jv, 1:-1]
    up[1:-1, 1:-1, 1:-1] = u[1:-1, jc, 1:-1]
    wp[1:-1, 1:-1, 1:-1] = w[1:-1, jc, 1:-1]
    for f in (up, vp, wp):
        _wrap(f)
    su, sv, sw = tend(u, v, w, c)
    sup, svp, swp = tend(up, vp, wp, c)
    d = max(np.abs(svp[1:-1, 1:-1, 1:-1] + sv[1:-1, jv, 1:-1]).max(),
            np.abs(sup[1:-1, 1:-1, 1:-1] - su[1:-1, jc, 1:-1]).max(),
            np.abs(swp[1:-1, 1:-1, 1:-1] - sw[1:-1, jc, 1:-1]).max())
    return float(d)


def pin_quadratic(tend):
    """s(2q) = 4 s(q) bit for bit (scaling by powers of two is exact)."""
    nx, ny, nz = 5, 4, 6
    c = inputs.make_coeffs(nz)
    u, v, w = _rand_periodic(nx, ny, nz, seed=17)
    s1 = tend(u, v, w, c)
    s2 = tend(2 * u, 2 * v, 2 * w, c)
    return float(max(np.abs(b - 4 * a).max() for a, b in zip(s1, s2)))


def pin_zhalo(tend):
    """The z-halo planes k = 0 and nz+1 are never read: filling them with NaN
    changes nothing."""
    nx, ny, nz = 5, 4, 6
    c = inputs.make_coeffs(nz)
    u, v, w = _rand_periodic(nx, ny, nz, seed=19)
    s1 = tend(u, v, w, c)
    u2, v2, w2 = (f.copy() for f in (u, v, w))
    for f in (u2, v2, w2):
        f[0] = np.nan
        f[nz + 1] = np.nan
    s2 = tend(u2, v2, w2, c)
    d = 0.0
    for a, b in zip(s1, s2):
        ia = a[1:-1, 1:-1, 1:-1]
        ib = b[1:-1, 1:-1, 1:-1]
        if not np.all(np.isfinite(ib)):
            return float("inf")
        d = max(d, float(np.abs(ia - ib).max()))
    return d


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


def pin_golden(tend):
    """Closed-form fixture tests/golden/linear_closed_form.json: exact rational
    values of the continuous operator for integer-coefficient linear fields."""
    g = load_golden("linear_closed_form.json")
    nx, ny, nz = g["nx"], g["ny"], g["nz"]
    dx, dy, dz = g["dx"], g["dy"], g["dz"]
    A = np.array(g["A"], dtype=np.float64)
    c, (u, v, w), _, _, _ = _linear_case(nx, ny, nz, dx, dy, dz, A)
    s = tend(u, v, w, c)
    err = 0.0
    for q, name in enumerate(("su", "sv", "sw")):
        for (k, j, i), num, den in g[name]:
            err = max(err, abs(s[q][k, j, i] - num / den) / max(1.0, abs(num / den)))
    return err


ALL = {
    "uniform_zero": pin_uniform_zero,
    "linear_exact": pin_linear_exact,
    "convergence": pin_convergence,
    "energy": pin_energy,
    "energy_anelastic": pin_energy_anelastic,
    "mirror_x": pin_mirror_x,
    "mirror_y": pin_mirror_y,
    "quadratic": pin_quadratic,
    "zhalo": pin_zhalo,
    "golden": pin_golden,
}


def failures(tend):
    """Names of the checks `tend` fails (exceptions count as failures)."""
    bad = []
    for name, fn in ALL.items():
        try:
            e = fn(tend)
        except Exception:            # a broken variant may produce garbage shapes
            bad.append(name)
            continue
        if not (e <= TOL[name]):
            bad.append(name)
    return bad
