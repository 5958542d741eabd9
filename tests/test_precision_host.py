"""Host logic of reduced-precision storage (no GPU): scales are powers of two,
keep FP16 values in range, and the a priori tendency bound holds."""
import math

import numpy as np

import oracle
from paper_2301_13016_gb300 import inputs, precision


def _is_pow2(x):
    m, _ = math.frexp(x)
    return m == 0.5


def test_scales_are_powers_of_two_and_in_range():
    c = inputs.make_coeffs(64)
    for maxabs in ((10.0, 10.0, 3.0), (1e-3, 5.0, 1e4), (0.7, 0.7, 0.7)):
        s = precision.suggest_scales(maxabs, c, "f16")
        assert all(_is_pow2(x) for x in s)
        for m, sin in zip(maxabs, s[:3]):
            assert m / sin <= 2 ** 14 and m / sin > 2 ** 12
        b = precision.tendency_bound(max(maxabs), c)
        assert b * s[3] <= 2 ** 15
    assert precision.suggest_scales((10, 10, 10), c, "bf16") == (1.0,) * 6


def test_tendency_bound_holds():
    nx, ny, nz = 16, 12, 10
    c = inputs.make_coeffs(nz)
    f = [x.numpy().astype(np.float64) for x in inputs.random_fields(nx, ny, nz)]
    m = max(np.abs(x).max() for x in f)
    s = oracle.tendencies(*f, c)
    a = oracle.abs_terms(*f, c)
    b = precision.tendency_bound(m, c)
    assert max(np.abs(x).max() for x in a) <= b
    assert max(np.abs(x).max() for x in s) <= b
