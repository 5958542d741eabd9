"""Seeded synthetic inputs for the PW advection scheme.

Shared by the tests, the benchmark and both sides of every parity check (the
CPU oracle and the CUDA library).  Holds none of the scheme's arithmetic: it
draws velocity fields, copies periodic halo values by indexing, and builds the
grid coefficients that are inputs of the scheme (tcx = 1/(4 dx), tcy = 1/(4 dy)
and the per-level vertical coefficients from a stretched column of levels).

Workload recipe (the paper's own problem is synthetic, "67 million grid
points", Sec. 5 Tables 1-2, with no published data):
  * u, v, w ~ amp * N(0, 1), amp = 10 m/s, drawn per field from
    torch.Generator seeds 2301, 2302, 2303;
  * w = 0 on the surface (k = 1) and the lid (k = nz);
  * doubly periodic lateral halo; z-halo planes (k = 0, nz+1) set to `zhalo`
    (never read by the scheme);
  * dx = dy = 100 m; level spacing stretched linearly from 20 m at the surface
    to 200 m at the lid;
  * smooth variant: 8 random sine modes per field, integer wavenumbers 1..8
    per periodic direction, vertical shape cos (u, v) or sin (w) with vertical
    wavenumber 1 or 2, normalised to max |q| = amp.

Field arrays are torch float32 tensors in the dense (nz+2, ny+2, nx+2) layout.
"""
from dataclasses import dataclass, field

import numpy as np
import torch

SEED_U, SEED_V, SEED_W = 2301, 2302, 2303


@dataclass
class Coeffs:
    """Grid coefficients of the PW scheme (inputs of the scheme).

    tcx, tcy: horizontal scalars; tzc1, tzc2 (u and v levels), tzd1, tzd2
    (w levels): float64 arrays of length nz+2 indexed by k; entries the scheme
    never uses are 0.  z_w (w levels), z_u (u/v levels), dz_u, dz_w and the
    reference densities rho_u, rho_w are kept for the invariant checks.
    """
    tcx: float
    tcy: float
    tzc1: np.ndarray
    tzc2: np.ndarray
    tzd1: np.ndarray
    tzd2: np.ndarray
    z_w: np.ndarray = field(repr=False, default=None)
    z_u: np.ndarray = field(repr=False, default=None)
    dz_u: np.ndarray = field(repr=False, default=None)
    dz_w: np.ndarray = field(repr=False, default=None)
    rho_u: np.ndarray = field(repr=False, default=None)
    rho_w: np.ndarray = field(repr=False, default=None)

    def as_dict(self):
        return dict(tcx=self.tcx, tcy=self.tcy, tzc1=self.tzc1, tzc2=self.tzc2,
                    tzd1=self.tzd1, tzd2=self.tzd2)


def levels(nz, dz_bottom=20.0, dz_top=200.0, uniform_dz=None):
    """w levels z_w[k] (k = 1..nz, z_w[1] = 0) and u levels z_u[k] (layer mid
    points, z_u[1] = -z_u[2]); arrays of length nz+2, entries 0 and nz+1
    extrapolated by one spacing."""
    if nz < 3:
        raise ValueError("nz must be >= 3")
    z_w = np.zeros(nz + 2)
    for k in range(2, nz + 1):
        if uniform_dz is not None:
            d = float(uniform_dz)
        else:
            d = dz_bottom + (dz_top - dz_bottom) * (k - 2) / (nz - 2)
        z_w[k] = z_w[k - 1] + d
    z_w[0] = -(z_w[2] - z_w[1])
    z_w[nz + 1] = z_w[nz] + (z_w[nz] - z_w[nz - 1])
    z_u = np.zeros(nz + 2)
    z_u[1:] = 0.5 * (z_w[:-1] + z_w[1:])
    z_u[1] = -z_u[2]
    z_u[0] = 2 * z_u[1] - z_u[2]
    return z_w, z_u


def make_coeffs(nz, dx=100.0, dy=100.0, dz_bottom=20.0, dz_top=200.0,
                uniform_dz=None, anelastic=False, scale_height=8000.0):
    """Coefficients for the default Boussinesq column (tzc1 = tzc2 = 1/(4 dz_u),
    tzd1 = tzd2 = 1/(4 dz_w)), or the anelastic one with a reference density
    exp(-z / scale_height) weighting the vertical fluxes."""
    z_w, z_u = levels(nz, dz_bottom, dz_top, uniform_dz)
    dz_u = np.zeros(nz + 2)
    dz_w = np.zeros(nz + 2)
    dz_u[2:nz + 1] = z_w[2:nz + 1] - z_w[1:nz]          # layer k spans z_w[k-1]..z_w[k]
    dz_w[1:nz] = z_u[2:nz + 1] - z_u[1:nz]              # w level k spans z_u[k]..z_u[k+1]
    if anelastic:
        rho_u = np.exp(-z_u / scale_height)
        rho_w = np.exp(-z_w / scale_height)
    else:
        rho_u = np.ones(nz + 2)
        rho_w = np.ones(nz + 2)
    tzc1 = np.zeros(nz + 2)
    tzc2 = np.zeros(nz + 2)
    tzd1 = np.zeros(nz + 2)
    tzd2 = np.zeros(nz + 2)
    for k in range(2, nz + 1):
        tzc1[k] = 0.25 * rho_w[k - 1] / (rho_u[k] * dz_u[k])
        tzc2[k] = 0.25 * rho_w[k] / (rho_u[k] * dz_u[k])
    for k in range(2, nz):
        tzd1[k] = 0.25 * rho_u[k] / (rho_w[k] * dz_w[k])
        tzd2[k] = 0.25 * rho_u[k + 1] / (rho_w[k] * dz_w[k])
    return Coeffs(tcx=0.25 / dx, tcy=0.25 / dy, tzc1=tzc1, tzc2=tzc2, tzd1=tzd1, tzd2=tzd2,
                  z_w=z_w, z_u=z_u, dz_u=dz_u, dz_w=dz_w, rho_u=rho_u, rho_w=rho_w)


def wrap_halo_(f):
    """Copy periodic images into the lateral halo of a dense (nz+2, ny+2, nx+2)
    tensor, in place, levels 1..nz (index copies only)."""
    nx, ny = f.shape[2] - 2, f.shape[1] - 2
    f[1:-1, 1:-1, 0] = f[1:-1, 1:-1, nx]
    f[1:-1, 1:-1, nx + 1] = f[1:-1, 1:-1, 1]
    f[1:-1, 0, :] = f[1:-1, ny, :]
    f[1:-1, ny + 1, :] = f[1:-1, 1, :]
    return f


def _gen(seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def random_fields(nx, ny, nz, amp=10.0, seeds=(SEED_U, SEED_V, SEED_W), device="cpu",
                  zhalo=0.0, lid=True):
    """u, v, w = amp * N(0,1) (float32), w = 0 at k = 1 and nz when lid is set,
    periodic lateral halo, z-halo planes = zhalo."""
    out = []
    for idx, seed in enumerate(seeds):
        f = torch.empty((nz + 2, ny + 2, nx + 2), dtype=torch.float32, device=device)
        f[1:-1, 1:-1, 1:-1] = torch.randn((nz, ny, nx), generator=_gen(seed, device),
                                          dtype=torch.float32, device=device) * amp
        if idx == 2 and lid:
            f[1] = 0.0
            f[nz] = 0.0
        wrap_halo_(f)
        f[0] = zhalo
        f[nz + 1] = zhalo
        out.append(f)
    return tuple(out)


def smooth_fields(nx, ny, nz, amp=10.0, nmodes=8, seeds=(SEED_U, SEED_V, SEED_W), device="cpu",
                  w_zero=False, zhalo=0.0):
    """Sum of nmodes random sine modes per field (float32), periodic in x and y,
    vertical shape cos(pi*kz*(k-1)/(nz-1)) for u, v and sin(...) for w (so w = 0
    at k = 1 and nz), normalised to max |q| = amp.  w_zero gives w = 0 everywhere."""
    out = []
    ii = torch.arange(1, nx + 1, dtype=torch.float64, device=device)
    jj = torch.arange(1, ny + 1, dtype=torch.float64, device=device)
    kk = torch.arange(1, nz + 1, dtype=torch.float64, device=device)
    for idx, seed in enumerate(seeds):
        g = _gen(seed, "cpu")
        kx = torch.randint(1, 9, (nmodes,), generator=g)
        ky = torch.randint(1, 9, (nmodes,), generator=g)
        kz = torch.randint(1, 3, (nmodes,), generator=g)
        ph = torch.rand((nmodes,), generator=g, dtype=torch.float64) * 2 * np.pi
        a = torch.rand((nmodes,), generator=g, dtype=torch.float64) + 0.5
        acc = torch.zeros((nz, ny, nx), dtype=torch.float64, device=device)
        for m in range(nmodes):
            horiz = torch.sin(2 * np.pi * (kx[m].item() * ii[None, :] / nx + ky[m].item() * jj[:, None] / ny)
                              + ph[m].item())
            arg = np.pi * kz[m].item() * (kk - 1) / (nz - 1)
            vert = torch.sin(arg) if idx == 2 else torch.cos(arg)
            acc += a[m].item() * vert[:, None, None] * horiz[None, :, :]
        if idx == 2:
            acc[0] = 0.0
            acc[nz - 1] = 0.0
        peak = acc.abs().max()
        if idx == 2 and w_zero:
            acc.zero_()
        elif peak > 0:
            acc *= amp / peak
        f = torch.empty((nz + 2, ny + 2, nx + 2), dtype=torch.float32, device=device)
        f[1:-1, 1:-1, 1:-1] = acc.to(torch.float32)
        wrap_halo_(f)
        f[0] = zhalo
        f[nz + 1] = zhalo
        out.append(f)
    return tuple(out)


def target_field(nx, ny, nz, std=10.0, seed=2305, device="cpu"):
    """Rollout target u_target ~ N(0, std^2) (float32), dense layout, zero halo."""
    f = torch.zeros((nz + 2, ny + 2, nx + 2), dtype=torch.float32, device=device)
    f[1:-1, 1:-1, 1:-1] = torch.randn((nz, ny, nx), generator=_gen(seed, device),
                                      dtype=torch.float32, device=device) * std
    return f


def batch_shapes(n=512, seed=2304, nxy=(32, 384), nzr=(32, 128), step=4):
    """Shapes (nx, ny, nz) of a batch of independent grids: nx, ny uniform in
    nxy with the given step, nz uniform in nzr."""
    g = _gen(seed, "cpu")
    lo, hi = nxy
    nxs = torch.randint(lo // step, hi // step + 1, (n,), generator=g) * step
    nys = torch.randint(lo // step, hi // step + 1, (n,), generator=g) * step
    nzs = torch.randint(nzr[0], nzr[1] + 1, (n,), generator=g)
    return [(int(a), int(b), int(c)) for a, b, c in zip(nxs, nys, nzs)]
