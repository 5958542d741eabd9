"""Helpers for the GPU tests (no tests here): set up a grid, move the seeded
dense fields into the library's layout, run the CUDA path, compare with the
oracle."""
import numpy as np
import torch

import paper_2301_13016_gb300 as pwlib
from paper_2301_13016_gb300 import inputs

NAN = float("nan")


def setup(nx, ny, nz, smooth=False, dtype="f32", grid=None, coeffs=None, zhalo=0.0, fields=None):
    c = coeffs if coeffs is not None else inputs.make_coeffs(nz)
    if fields is None:
        gen = inputs.smooth_fields if smooth else inputs.random_fields
        fields = gen(nx, ny, nz, zhalo=zhalo)
    g = grid if grid is not None else pwlib.Grid(nx, ny, nz, dtype=dtype)
    h = pwlib.PW(g, c)
    dev = [g.from_dense(f) for f in fields]
    outs = [g.alloc(fill=NAN) for _ in range(3)]
    return c, fields, g, h, dev, outs


def dense_out(g, outs, scale=(1.0, 1.0, 1.0)):
    return [g.to_dense(o, s).numpy() for o, s in zip(outs, scale)]


def interior(a):
    return a[1:-1, 1:-1, 1:-1]


def rel_errs(got, ref):
    """max|got - ref| / max|ref| per field over interior cells."""
    return [float(np.abs(interior(a) - interior(b)).max() / max(np.abs(interior(b)).max(), 1e-300))
            for a, b in zip(got, ref)]


def run(h, dev, outs, **kw):
    h.tendencies(*dev, *outs, **kw)
    h.sync()
    torch.cuda.synchronize()
