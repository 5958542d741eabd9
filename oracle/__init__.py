"""CPU oracle for the Piacsek-Williams advection scheme (Sec. 2.2, Sec. 4).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only tests/, the smoke check and the
benchmark's CPU-baseline leg and reference arm import this package.  It shares no code with the
CUDA library (paper_2301_13016_gb300) and imports nothing from it.

Thin ctypes wrapper over oracle/pw_oracle.c (plain C loop nests, FP64 and FP32).
Arrays are numpy, in the oracle's dense layout: shape (nz+2, ny+2, nx+2), one
halo cell on every side, C order.  Coefficients are any object (or mapping)
with tcx, tcy (scalars) and tzc1, tzc2, tzd1, tzd2 (length nz+2, indexed by k).

Parity status of each function (what pins it, see tests/test_oracle_pins.py):
  tendencies            pinned: uniform-flow zero, exact result for linear
                        fields (continuous skew-symmetric form), second-order
                        convergence, discrete energy identity, mirror
                        antisymmetry, golden closed-form fixture.
  fill_halo_periodic    pinned: numpy wrap padding.
  step                  pinned: energy growth identity of forward Euler,
                        agreement with repeated (fill, tendencies, update).
  adjoint_tendencies    pinned: dot-product test against the linearisation
                        J(q)d = s(q+d) - s(q) - s(d) of the pinned tendencies.
  fold_halo_periodic    pinned: dot-product test against fill_halo_periodic.
  step_adjoint          pinned: central finite differences of a rollout loss.
  abs_terms             pinned: triangle inequality (>= |tendency|), equality
                        for single-term inputs, quadratic scaling, and the
                        observed rounding error of the FP32 oracle stays
                        inside the bound it gives.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i = ctypes.c_int
        lib.pw_oracle_tendencies_f64.argtypes = [i, i, i, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                                 _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        lib.pw_oracle_tendencies_f64.restype = None
        lib.pw_oracle_tendencies_f32.argtypes = [i, i, i, _fp, _fp, _fp, ctypes.c_float, ctypes.c_float,
                                                 _fp, _fp, _fp, _fp, _fp, _fp, _fp]
        lib.pw_oracle_tendencies_f32.restype = None
        lib.pw_oracle_fill_halo_periodic_f64.argtypes = [i, i, i, _dp]
        lib.pw_oracle_fill_halo_periodic_f64.restype = None
        lib.pw_oracle_fill_halo_periodic_f32.argtypes = [i, i, i, _fp]
        lib.pw_oracle_fill_halo_periodic_f32.restype = None
        lib.pw_oracle_step_f64.argtypes = [i, i, i, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                           _dp, _dp, _dp, _dp, ctypes.c_double, i]
        lib.pw_oracle_step_f64.restype = ctypes.c_int
        lib.pw_oracle_adjoint_tendencies_f64.argtypes = [i, i, i, _dp, _dp, _dp, ctypes.c_double,
                                                         ctypes.c_double, _dp, _dp, _dp, _dp,
                                                         _dp, _dp, _dp, _dp, _dp, _dp]
        lib.pw_oracle_adjoint_tendencies_f64.restype = None
        lib.pw_oracle_fold_halo_periodic_f64.argtypes = [i, i, i, _dp]
        lib.pw_oracle_fold_halo_periodic_f64.restype = None
        lib.pw_oracle_step_adjoint_f64.argtypes = [i, i, i, _dp, _dp, _dp, ctypes.c_double,
                                                   ctypes.c_double, _dp, _dp, _dp, _dp,
                                                   ctypes.c_double, i, _dp, _dp, _dp]
        lib.pw_oracle_step_adjoint_f64.restype = ctypes.c_int
        lib.pw_oracle_abs_terms_f64.argtypes = [i, i, i, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                                _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        lib.pw_oracle_abs_terms_f64.restype = None
        _LIB = lib
    return _LIB


def _get(c, name):
    return c[name] if isinstance(c, dict) else getattr(c, name)


def _shape(f):
    nz, ny, nx = (s - 2 for s in f.shape)
    return nx, ny, nz


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a, ct):
    return a.ctypes.data_as(ct)


def _coeffs(c, dtype, nz):
    tz = [_arr(_get(c, n), dtype) for n in ("tzc1", "tzc2", "tzd1", "tzd2")]
    for t in tz:
        if t.shape != (nz + 2,):
            raise ValueError("vertical coefficient arrays must have length nz+2")
    return dtype(_get(c, "tcx")), dtype(_get(c, "tcy")), tz


def tendencies(u, v, w, coeffs, precision="f64"):
    """Source terms (su, sv, sw) of the PW scheme; halo cells of the result are 0.

    precision "f64": inputs upcast to float64, arithmetic in float64.
    precision "f32": inputs, coefficients and arithmetic in float32, evaluated
    in the written order without fused multiply-add.
    """
    dtype = {"f64": np.float64, "f32": np.float32}[precision]
    ct = _dp if dtype is np.float64 else _fp
    u, v, w = (_arr(a, dtype) for a in (u, v, w))
    if not (u.shape == v.shape == w.shape) or u.ndim != 3:
        raise ValueError("u, v, w must share one (nz+2, ny+2, nx+2) shape")
    nx, ny, nz = _shape(u)
    tcx, tcy, tz = _coeffs(coeffs, dtype, nz)
    su, sv, sw = (np.zeros_like(u) for _ in range(3))
    fn = _lib().pw_oracle_tendencies_f64 if dtype is np.float64 else _lib().pw_oracle_tendencies_f32
    fn(nx, ny, nz, _ptr(u, ct), _ptr(v, ct), _ptr(w, ct), tcx, tcy,
       *[_ptr(t, ct) for t in tz], _ptr(su, ct), _ptr(sv, ct), _ptr(sw, ct))
    return su, sv, sw


def fill_halo_periodic(f, precision="f64"):
    """Return a copy of f with its lateral halo filled periodically (levels 1..nz)."""
    dtype = {"f64": np.float64, "f32": np.float32}[precision]
    g = np.array(f, dtype=dtype, copy=True, order="C")
    nx, ny, nz = _shape(g)
    if dtype is np.float64:
        _lib().pw_oracle_fill_halo_periodic_f64(nx, ny, nz, _ptr(g, _dp))
    else:
        _lib().pw_oracle_fill_halo_periodic_f32(nx, ny, nz, _ptr(g, _fp))
    return g


def step(u, v, w, coeffs, dt, nsteps):
    """nsteps forward-Euler steps q <- q + dt*s(q) in float64; returns new (u, v, w)
    with periodic halos filled."""
    u, v, w = (np.array(a, dtype=np.float64, copy=True, order="C") for a in (u, v, w))
    nx, ny, nz = _shape(u)
    tcx, tcy, tz = _coeffs(coeffs, np.float64, nz)
    rc = _lib().pw_oracle_step_f64(nx, ny, nz, _ptr(u, _dp), _ptr(v, _dp), _ptr(w, _dp), tcx, tcy,
                                   *[_ptr(t, _dp) for t in tz], float(dt), int(nsteps))
    if rc != 0:
        raise MemoryError("oracle step: allocation failed")
    return u, v, w


def adjoint_tendencies(u, v, w, coeffs, lsu, lsv, lsw):
    """J(u,v,w)^T [lsu; lsv; lsw] on the full padded arrays (halo entries are the
    sensitivities to the halo inputs), float64."""
    u, v, w, lsu, lsv, lsw = (_arr(a, np.float64) for a in (u, v, w, lsu, lsv, lsw))
    nx, ny, nz = _shape(u)
    tcx, tcy, tz = _coeffs(coeffs, np.float64, nz)
    gu, gv, gw = (np.zeros_like(u) for _ in range(3))
    _lib().pw_oracle_adjoint_tendencies_f64(nx, ny, nz, _ptr(u, _dp), _ptr(v, _dp), _ptr(w, _dp), tcx, tcy,
                                            *[_ptr(t, _dp) for t in tz],
                                            _ptr(lsu, _dp), _ptr(lsv, _dp), _ptr(lsw, _dp),
                                            _ptr(gu, _dp), _ptr(gv, _dp), _ptr(gw, _dp))
    return gu, gv, gw


def fold_halo_periodic(g):
    """Transpose of fill_halo_periodic: returns a copy with halo sensitivities
    added to their interior images and the lateral halo cleared (levels 1..nz)."""
    g = np.array(g, dtype=np.float64, copy=True, order="C")
    nx, ny, nz = _shape(g)
    _lib().pw_oracle_fold_halo_periodic_f64(nx, ny, nz, _ptr(g, _dp))
    return g


def step_adjoint(u0, v0, w0, coeffs, dt, nsteps, gu, gv, gw):
    """dL/dq at the start of an nsteps forward-Euler rollout from (u0, v0, w0),
    given dL/dq (gu, gv, gw) at its end.  Interior entries; halos zero."""
    u0, v0, w0 = (_arr(a, np.float64) for a in (u0, v0, w0))
    gu, gv, gw = (np.array(a, dtype=np.float64, copy=True, order="C") for a in (gu, gv, gw))
    nx, ny, nz = _shape(u0)
    tcx, tcy, tz = _coeffs(coeffs, np.float64, nz)
    rc = _lib().pw_oracle_step_adjoint_f64(nx, ny, nz, _ptr(u0, _dp), _ptr(v0, _dp), _ptr(w0, _dp),
                                           tcx, tcy, *[_ptr(t, _dp) for t in tz], float(dt), int(nsteps),
                                           _ptr(gu, _dp), _ptr(gv, _dp), _ptr(gw, _dp))
    if rc != 0:
        raise MemoryError("oracle step_adjoint: allocation failed")
    return gu, gv, gw


def abs_terms(u, v, w, coeffs):
    """Per-cell sum over the scheme's terms c*a*(b+d) of |c|*|a|*(|b|+|d|)
    (float64; zero where the scheme writes zero): the magnitude that running
    error bounds of the scheme scale with."""
    u, v, w = (_arr(a, np.float64) for a in (u, v, w))
    nx, ny, nz = _shape(u)
    tcx, tcy, tz = _coeffs(coeffs, np.float64, nz)
    au, av, aw = (np.zeros_like(u) for _ in range(3))
    _lib().pw_oracle_abs_terms_f64(nx, ny, nz, _ptr(u, _dp), _ptr(v, _dp), _ptr(w, _dp), tcx, tcy,
                                   *[_ptr(t, _dp) for t in tz], _ptr(au, _dp), _ptr(av, _dp), _ptr(aw, _dp))
    return au, av, aw


def library_path():
    return _build.LIB


__all__ = ["tendencies", "fill_halo_periodic", "step", "adjoint_tendencies",
           "fold_halo_periodic", "step_adjoint", "abs_terms", "library_path"]
