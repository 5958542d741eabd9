"""Reduced-precision storage: unit roundoffs and per-field power-of-two scales.

Fields may be stored in HBM as BF16 or FP16 with FP32 arithmetic; the C ABI
takes six scales {in_u, in_v, in_w, out_su, out_sv, out_sw}: physical input =
stored * in, stored output = physical * out.  Powers of two keep the scaling
exact, so it only moves values within the format's exponent range.
"""
import math

UNIT_ROUNDOFF = {"f32": 2.0 ** -24, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}
# smallest positive normal number of each storage format
MIN_NORMAL = {"f32": 2.0 ** -126, "bf16": 2.0 ** -126, "f16": 2.0 ** -14}
# largest stored magnitude the scales aim for (well inside the format's range)
TARGET_MAX = {"f32": None, "bf16": None, "f16": 2.0 ** 14}


def _pow2_at_least(x):
    return 2.0 ** math.ceil(math.log2(x)) if x > 0 else 1.0


def tendency_bound(maxabs, coeffs):
    """A priori bound on |su|, |sv|, |sw| for inputs with max |q| <= maxabs:
    every output is a sum of at most six terms c*a*(b+d) with |a|, |b|, |d| <=
    maxabs (two x-terms, two y-terms, two z-terms)."""
    get = (lambda n: coeffs[n]) if isinstance(coeffs, dict) else (lambda n: getattr(coeffs, n))
    tz = max(max(abs(float(x)) for x in get(n)) for n in ("tzc1", "tzc2", "tzd1", "tzd2"))
    cx, cy = abs(float(get("tcx"))), abs(float(get("tcy")))
    return 2.0 * maxabs * maxabs * (2 * cx + 2 * cy + 2 * tz)


def suggest_scales(maxabs, coeffs, dtype):
    """Scales {in_u, in_v, in_w, out_su, out_sv, out_sw} for fields with
    max |u|, |v|, |w| <= maxabs[0..2].  FP16: stored inputs stay <= 2^14 and
    stored outputs <= 2^15 (max finite 65504); BF16 and FP32 share FP32's
    exponent range and need no scaling (all ones)."""
    if dtype in ("f32", "bf16"):
        return (1.0,) * 6
    if dtype != "f16":
        raise ValueError("dtype must be f32, bf16 or f16")
    ins = tuple(_pow2_at_least(m) / TARGET_MAX["f16"] for m in maxabs)
    b = tendency_bound(max(maxabs), coeffs)
    out = TARGET_MAX["f16"] * 2.0 / _pow2_at_least(b)
    return ins + (out, out, out)
