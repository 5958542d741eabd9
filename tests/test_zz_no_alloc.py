"""pw_weighted_dot_noalloc: the allocation-free weighted inner product.

Callers that cannot call cudaMalloc once their run has started (a host model
that owns the device memory budget, a time loop that must not meet an
allocation failure) use this entry point: it keeps its scratch in the
library's static device array.  Checked through the C ABI against
pw_weighted_dot on the same fields, twice in a row (the second call reuses
the array the first one left behind).  This file sorts last so that a run
stopping at its first failure has run every other test before it.
"""
import numpy as np
import pytest
import torch

import paper_2301_13016_gb300 as pwlib
from paper_2301_13016_gb300 import inputs

pytestmark = pytest.mark.gpu


def _fields(nx, ny, nz, seed):
    c = inputs.make_coeffs(nz, anelastic=True)
    f = inputs.random_fields(nx, ny, nz, seeds=(seed, seed + 1, seed + 2))
    g = pwlib.Grid(nx, ny, nz)
    h = pwlib.PW(g, c)
    dev = [g.from_dense(x) for x in f]
    outs = [g.alloc() for _ in range(3)]
    h.tendencies(*dev, *outs)
    h.sync()
    return c, g, h, dev, outs


def test_noalloc_dot_matches_allocating_dot_twice():
    c, g, h, dev, outs = _fields(256, 40, 24, 11)
    wu = c.rho_u * c.dz_u
    cases = [(dev[0], outs[0], wu, 2, g.nz), (dev[1], dev[1], None, 1, g.nz),
             (dev[2], outs[2], c.rho_w * c.dz_w, 2, g.nz - 1)]
    for a, b, wk, k0, k1 in cases:
        ref = h.weighted_dot(a, b, wk=wk, k0=k0, k1=k1)
        first = h.weighted_dot_noalloc(a, b, wk=wk, k0=k0, k1=k1)
        second = h.weighted_dot_noalloc(a, b, wk=wk, k0=k0, k1=k1)
        scale = h.weighted_dot(a, a, wk=None if wk is None else np.abs(wk), k0=k0, k1=k1)
        # same kernels, same block count on this GPU: identical up to the order
        # of a fixed reduction, so agreement to rounding of the scale
        assert abs(first - ref) <= 1e-12 * max(abs(scale), 1.0)
        assert abs(second - ref) <= 1e-12 * max(abs(scale), 1.0)


def test_noalloc_dot_other_grid_and_limit():
    # a second handle and grid size on the same device share the array
    c, g, h, dev, outs = _fields(128, 12, 9, 21)
    ref = h.weighted_dot(dev[0], outs[0], wk=c.dz_u, k0=2, k1=g.nz)
    got = h.weighted_dot_noalloc(dev[0], outs[0], wk=c.dz_u, k0=2, k1=g.nz)
    assert got == pytest.approx(ref, rel=1e-12, abs=1e-12)
    # grids deeper than the static array's level limit are rejected, not truncated
    nz = 4095
    g2 = pwlib.Grid(4, 4, nz)
    h2 = pwlib.PW(g2, inputs.make_coeffs(nz))
    t = g2.alloc()
    with pytest.raises(pwlib.PwError) as e:
        h2.weighted_dot_noalloc(t, t, wk=np.ones(nz + 2))
    assert e.value.status == pwlib.PW_ERR_UNSUPPORTED
    assert "4096" in str(e.value)


def test_noalloc_first_call_leaves_free_memory_unchanged():
    """The property the entry point exists for: on a fresh handle, its first
    call leaves the device's free memory exactly as it was, while the
    allocating pw_weighted_dot's first call on a fresh handle takes its
    scratch from the device (here 2.4 MB, so at least one new 2 MiB page)."""
    c, g, h0, dev, outs = _fields(128, 16, 12, 31)
    wk = c.dz_u
    # the library's device code, the static array with it, is loaded by the
    # first call in the process; measure from the second handle on
    ref = h0.weighted_dot_noalloc(dev[0], outs[0], wk=wk, k0=2, k1=g.nz)
    torch.cuda.synchronize()
    h1 = pwlib.PW(g, c)
    free0 = torch.cuda.mem_get_info()[0]
    got = h1.weighted_dot_noalloc(dev[0], outs[0], wk=wk, k0=2, k1=g.nz)
    again = h1.weighted_dot_noalloc(dev[0], outs[0], wk=wk, k0=2, k1=g.nz)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert got == ref and again == ref

    # positive control: the same measurement sees the allocating entry point's
    # scratch (4 * (blocks + 1) + nz + 2 doubles; nz = 300000 makes it 2.4 MB)
    nz = 300_000
    gd = pwlib.Grid(4, 4, nz, pitch_j=8, pitch_k=48, origin=9)
    hd = pwlib.PW(gd, inputs.make_coeffs(nz))
    t = gd.alloc(fill=1.0)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    val = hd.weighted_dot(t, t)
    torch.cuda.synchronize()
    assert free1 - torch.cuda.mem_get_info()[0] >= 2 * 1024 * 1024
    assert val == pytest.approx(4 * 4 * nz, rel=1e-12)
