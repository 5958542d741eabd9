"""Python binding of libpw.so (the C ABI in include/pw.h).

Argument marshalling only: every step of the scheme runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if libpw.so is missing or cannot be loaded, every call raises.

Fields are flat 1-D tensors holding one whole allocation of a Grid's layout
(Grid.alloc); Grid.view gives the (nz+2, ny+2*halo, nx+2*halo) strided view of
one.  Entry points keep the C names without the pw_ prefix.
"""
import ctypes
import os

import numpy as np
import torch

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG_DIR, "libpw.so")

PW_ADJ_ACCUMULATE, PW_ADJ_PERIODIC, PW_ADJ_ADD_LAMBDA = 1, 2, 4
PW_OK, PW_ERR_ARG, PW_ERR_ALIGN, PW_ERR_CUDA, PW_ERR_OOM, PW_ERR_DEVICE_TIMEOUT, PW_ERR_UNSUPPORTED = range(7)
DTYPES = {"f32": (0, torch.float32), "bf16": (1, torch.bfloat16), "f16": (2, torch.float16)}


class PwError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg}")
        self.status = status


class pw_grid_t(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("halo", ctypes.c_int32),
                ("pitch_j", ctypes.c_int64), ("pitch_k", ctypes.c_int64), ("origin", ctypes.c_int64),
                ("dtype", ctypes.c_int)]


_dp = ctypes.POINTER(ctypes.c_double)


class pw_coeffs_t(ctypes.Structure):
    _fields_ = [("tcx", ctypes.c_double), ("tcy", ctypes.c_double), ("tzc1", _dp), ("tzc2", _dp),
                ("tzd1", _dp), ("tzd2", _dp)]


# (name, restype, argtypes) of every exported entry point
_VP = ctypes.c_void_p
_I32 = ctypes.c_int32
_FP = ctypes.POINTER(ctypes.c_float)
SIGNATURES = [
    ("pw_grid_default", ctypes.c_int, [_I32, _I32, _I32, _I32, ctypes.c_int, ctypes.POINTER(pw_grid_t),
                                       ctypes.POINTER(ctypes.c_int64)]),
    ("pw_create", ctypes.c_int, [ctypes.POINTER(pw_grid_t), ctypes.POINTER(pw_coeffs_t), ctypes.POINTER(_VP)]),
    ("pw_destroy", ctypes.c_int, [_VP]),
    ("pw_set_kernel", ctypes.c_int, [_VP, _I32]),
    ("pw_set_tma_config", ctypes.c_int, [_VP, _I32, _I32, _I32, _I32, _I32, _I32]),
    ("pw_set_step_blocking", ctypes.c_int, [_VP, _I32, _I32, _I32, _I32, _I32]),
    ("pw_get_tma_config", ctypes.c_int, [_VP, _I32, ctypes.POINTER(_I32)]),
    ("pw_set_adjoint_config", ctypes.c_int, [_VP, _I32, _I32, _I32, _I32]),
    ("pw_get_adjoint_config", ctypes.c_int, [_VP, ctypes.POINTER(_I32)]),
    ("pw_tendencies", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _FP, _VP]),
    ("pw_tendencies_host", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _FP, _VP]),
    ("pw_tendencies_host_async", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _FP, _VP]),
    ("pw_fill_halo_periodic", ctypes.c_int, [_VP, _VP, _VP]),
    ("pw_adjoint", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_float, _I32, _VP]),
    ("pw_step", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_float, _I32, _FP, _VP]),
    ("pw_step_to", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_float, _FP, _VP]),
    ("pw_error_norms", ctypes.c_int, [_VP, _VP, ctypes.c_float, _VP, _I32, _I32, _dp, _VP]),
    ("pw_weighted_dot", ctypes.c_int, [_VP, _VP, ctypes.c_float, _VP, ctypes.c_float, _dp, _I32, _I32, _dp, _VP]),
    ("pw_weighted_dot_noalloc", ctypes.c_int, [_VP, _VP, ctypes.c_float, _VP, ctypes.c_float, _dp, _I32, _I32,
                                               _dp, _VP]),
    ("pw_sync", ctypes.c_int, [_VP, _VP]),
    ("pw_selftest_wait_timeout", ctypes.c_int, [_VP, ctypes.c_int64, _VP]),
    ("pw_inject_failures", ctypes.c_int, [_I32, _I32]),
    ("pw_debug_bounds_build", ctypes.c_int32, []),
    ("pw_debug_layout_check", ctypes.c_int32, [ctypes.POINTER(pw_grid_t), ctypes.c_int64, _I32, _I32]),
    ("pw_batch_create", ctypes.c_int, [_I32, ctypes.POINTER(pw_grid_t), ctypes.POINTER(pw_coeffs_t),
                                       ctypes.POINTER(_VP)]),
    ("pw_batch_set_config", ctypes.c_int, [_VP, _I32, _I32, _I32, _I32, _I32, _I32]),
    ("pw_batch_set_narrow_columns", ctypes.c_int, [_VP, _I32]),
    ("pw_batch_narrow_shape", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_int32)]),
    ("pw_batch_info", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(_I32)]),
    ("pw_batch_tendencies", ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                           ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP), _FP, _VP]),
    ("pw_batch_sync", ctypes.c_int, [_VP, _VP]),
    ("pw_batch_destroy", ctypes.c_int, [_VP]),
    ("pw_last_error", ctypes.c_char_p, []),
    ("pw_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("pw_last_kernel", _I32, [_VP]),
]

_LIB = None


def lib():
    """The loaded libpw.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _check(status, what):
    if status != PW_OK:
        msg = lib().pw_last_error().decode(errors="replace")
        name = lib().pw_status_string(status).decode()
        raise PwError(status, f"{what}: {name}: {msg}")


INJECT_ALLOC, INJECT_TENSOR_MAP = 0, 1


def inject_failures(kind, count):
    """Host-side failure injection for tests: the library's next `count`
    device or pinned allocations (INJECT_ALLOC) or TMA descriptor encodings
    (INJECT_TENSOR_MAP) fail as the CUDA call would; count 0 clears."""
    _check(lib().pw_inject_failures(int(kind), int(count)), "pw_inject_failures")


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Grid:
    """A grid and its field layout (pw_grid_t).  Default layout from
    pw_grid_default unless pitch_j, pitch_k, origin are all given."""

    def __init__(self, nx, ny, nz, halo=1, dtype="f32", pitch_j=None, pitch_k=None, origin=None):
        if dtype not in DTYPES:
            raise ValueError(f"dtype must be one of {list(DTYPES)}")
        self.dtype = dtype
        self.torch_dtype = DTYPES[dtype][1]
        if pitch_j is None:
            g = pw_grid_t()
            n = ctypes.c_int64()
            _check(lib().pw_grid_default(nx, ny, nz, halo, DTYPES[dtype][0], ctypes.byref(g), ctypes.byref(n)),
                   "pw_grid_default")
            self.c = g
            self.alloc_elems = int(n.value)
        else:
            self.c = pw_grid_t(nx, ny, nz, halo, pitch_j, pitch_k, origin, DTYPES[dtype][0])
            self.alloc_elems = int(origin + (nz + 1) * pitch_k + (ny + halo) * pitch_j + nx + halo + 1)
        self.nx, self.ny, self.nz, self.halo = nx, ny, nz, halo

    @property
    def pitch_j(self):
        return int(self.c.pitch_j)

    @property
    def pitch_k(self):
        return int(self.c.pitch_k)

    @property
    def origin(self):
        return int(self.c.origin)

    @property
    def cells(self):
        return self.nx * self.ny * self.nz

    def alloc(self, device="cuda", fill=0.0):
        t = torch.empty(self.alloc_elems, dtype=self.torch_dtype, device=device)
        if fill is not None:
            t.fill_(fill)
        return t

    def view(self, flat):
        """(nz+2, ny+2*halo, nx+2*halo) view of a flat allocation; index
        [k, j+halo-1, i+halo-1] is element (k, j, i)."""
        h = self.halo
        off = flat.storage_offset() + self.origin + (1 - h) * self.pitch_j + (1 - h)
        return torch.as_strided(flat, (self.nz + 2, self.ny + 2 * h, self.nx + 2 * h),
                                (self.pitch_k, self.pitch_j, 1), off)

    def from_dense(self, dense, device="cuda", scale=1.0):
        """New allocation holding a dense (nz+2, ny+2, nx+2) array (one halo
        cell); stored = value / scale in the grid's dtype."""
        t = self.alloc(device=device)
        src = torch.as_tensor(np.asarray(dense) if not torch.is_tensor(dense) else dense)
        if scale != 1.0:
            src = src.double() / scale
        h = self.halo
        self.view(t)[:, h - 1:h + self.ny + 1, h - 1:h + self.nx + 1].copy_(src.to(device=device,
                                                                                     dtype=self.torch_dtype))
        return t

    def to_dense(self, flat, scale=1.0):
        """Dense (nz+2, ny+2, nx+2) float64 CPU copy of a field (one halo cell)."""
        h = self.halo
        v = self.view(flat)[:, h - 1:h + self.ny + 1, h - 1:h + self.nx + 1]
        out = v.detach().to("cpu").double()
        return out * scale if scale != 1.0 else out


def _ptr(t, grid, what, host=False):
    """Address of a field allocation: a CUDA tensor (a CPU one for the host
    entry point, host=True), of the grid's dtype, flat and large enough."""
    if not torch.is_tensor(t):
        raise TypeError(f"{what} must be a torch tensor")
    if host == t.is_cuda:
        raise ValueError(f"{what} must be a {'host' if host else 'CUDA'} tensor (got {t.device})")
    if t.dtype != grid.torch_dtype:
        raise TypeError(f"{what} has dtype {t.dtype}, grid stores {grid.torch_dtype}")
    if t.dim() != 1 or not t.is_contiguous() or t.numel() < grid.alloc_elems:
        raise ValueError(f"{what} must be a flat contiguous allocation of >= {grid.alloc_elems} elements")
    return ctypes.c_void_p(t.data_ptr())


def _scale_arg(scale):
    if scale is None:
        return None
    arr = (ctypes.c_float * 6)(*[float(x) for x in scale])
    return ctypes.cast(arr, _FP), arr


class PW:
    """A pw_handle_t: one grid, one coefficient set, on the current device."""

    def __init__(self, grid, coeffs):
        self.grid = grid
        nz = grid.nz
        arrs = []
        for name in ("tzc1", "tzc2", "tzd1", "tzd2"):
            a = np.ascontiguousarray(getattr(coeffs, name) if not isinstance(coeffs, dict) else coeffs[name],
                                     dtype=np.float64)
            if a.shape != (nz + 2,):
                raise ValueError(f"{name} must have nz+2 = {nz + 2} entries")
            arrs.append(a)
        get = (lambda n: coeffs[n]) if isinstance(coeffs, dict) else (lambda n: getattr(coeffs, n))
        c = pw_coeffs_t(float(get("tcx")), float(get("tcy")), *[a.ctypes.data_as(_dp) for a in arrs])
        h = ctypes.c_void_p()
        _check(lib().pw_create(ctypes.byref(grid.c), ctypes.byref(c), ctypes.byref(h)), "pw_create")
        self.h = h
        self.device = torch.cuda.current_device()

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().pw_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_kernel(self, kind):
        _check(lib().pw_set_kernel(self.h, int(kind)), "pw_set_kernel")

    def set_tma_config(self, ty=0, stages=0, nseg=0, lanes_x=0, cells=0, rows=0):
        """Launch shape of the k-march kernel (0 = automatic); rows = rows per
        thread (2: packed FP32x2 arithmetic on row pairs, 16-bit storage;
        3: one row per thread, its cells packed as FP32x2 pairs along x,
        16-bit storage)."""
        _check(lib().pw_set_tma_config(self.h, int(lanes_x), int(cells), int(ty), int(stages), int(nseg),
                                       int(rows)), "pw_set_tma_config")

    def tma_config(self, step=False):
        """The k-march launch shape tendencies() (or step(), with step=True)
        uses: dict(lanes_x, cells, ty, stages, nseg, rows)."""
        out = (_I32 * 6)()
        _check(lib().pw_get_tma_config(self.h, 1 if step else 0, out), "pw_get_tma_config")
        return dict(zip(("lanes_x", "cells", "ty", "stages", "nseg", "rows"), list(out)))

    def set_adjoint_config(self, cells=0, ty=0, stages=0, nseg=0):
        """Launch shape of the TMA adjoint (0 = automatic): cells per thread
        along x, rows per CTA, ring slots, CTAs along z."""
        _check(lib().pw_set_adjoint_config(self.h, int(cells), int(ty), int(stages), int(nseg)),
               "pw_set_adjoint_config")

    def adjoint_config(self):
        """The TMA adjoint's launch shape: dict(cells, ty, stages, nseg)."""
        out = (_I32 * 4)()
        _check(lib().pw_get_adjoint_config(self.h, out), "pw_get_adjoint_config")
        return dict(zip(("cells", "ty", "stages", "nseg"), list(out)))

    def set_step_blocking(self, steps_per_pass=0, ty=0, stages=0, ctas_per_sm=0, nseg=0):
        """Temporal blocking of step(): 1 or 2 steps per kernel pass (0 =
        automatic = 1; 2 needs the TMA path and a halo >= 2), and the
        two-step kernel's launch shape (0 = automatic)."""
        _check(lib().pw_set_step_blocking(self.h, int(steps_per_pass), int(ty), int(stages), int(ctas_per_sm),
                                          int(nseg)), "pw_set_step_blocking")

    @property
    def last_kernel(self):
        return int(lib().pw_last_kernel(self.h))

    def tendencies(self, u, v, w, su, sv, sw, scale=None, stream=None):
        g = self.grid
        sp = _scale_arg(scale)
        _check(lib().pw_tendencies(self.h, _ptr(u, g, "u"), _ptr(v, g, "v"), _ptr(w, g, "w"), _ptr(su, g, "su"),
                                   _ptr(sv, g, "sv"), _ptr(sw, g, "sw"), sp[0] if sp else None,
                                   _stream_ptr(stream)), "pw_tendencies")

    def tendencies_host(self, u, v, w, su, sv, sw, scale=None, stream=None):
        """HOST tensors (pinned or pageable) in and out; synchronous."""
        g = self.grid
        sp = _scale_arg(scale)
        H = dict(host=True)
        _check(lib().pw_tendencies_host(self.h, _ptr(u, g, "u", **H), _ptr(v, g, "v", **H), _ptr(w, g, "w", **H),
                                        _ptr(su, g, "su", **H), _ptr(sv, g, "sv", **H), _ptr(sw, g, "sw", **H),
                                        sp[0] if sp else None, _stream_ptr(stream)), "pw_tendencies_host")

    def tendencies_host_async(self, u, v, w, su, sv, sw, scale=None, stream=None):
        """HOST tensors in and out, returns once enqueued: the outputs are
        ready after sync(stream); keep the tensors alive and unchanged until
        then (pinned memory for overlap)."""
        g = self.grid
        sp = _scale_arg(scale)
        H = dict(host=True)
        _check(lib().pw_tendencies_host_async(self.h, _ptr(u, g, "u", **H), _ptr(v, g, "v", **H),
                                              _ptr(w, g, "w", **H), _ptr(su, g, "su", **H), _ptr(sv, g, "sv", **H),
                                              _ptr(sw, g, "sw", **H), sp[0] if sp else None, _stream_ptr(stream)),
               "pw_tendencies_host_async")
        self._keep = (u, v, w, su, sv, sw, sp)   # alive until the next call

    def step(self, u, v, w, tmp_u, tmp_v, tmp_w, dt, nsteps, scale=None, stream=None):
        """nsteps forward-Euler steps in place on (u, v, w); tmp_* are scratch."""
        g = self.grid
        sp = None
        if scale is not None:
            arr = (ctypes.c_float * 3)(*[float(x) for x in scale])
            sp = (ctypes.cast(arr, _FP), arr)
        _check(lib().pw_step(self.h, _ptr(u, g, "u"), _ptr(v, g, "v"), _ptr(w, g, "w"), _ptr(tmp_u, g, "tmp_u"),
                             _ptr(tmp_v, g, "tmp_v"), _ptr(tmp_w, g, "tmp_w"), float(dt), int(nsteps),
                             sp[0] if sp else None, _stream_ptr(stream)), "pw_step")

    def step_to(self, u, v, w, nu, nv, nw, dt, scale=None, stream=None):
        """One forward-Euler step out of place: (nu, nv, nw) = q + dt*s(q) with
        the result's periodic halo; the halos of (u, v, w) must be periodic."""
        g = self.grid
        sp = None
        if scale is not None:
            arr = (ctypes.c_float * 3)(*[float(x) for x in scale])
            sp = (ctypes.cast(arr, _FP), arr)
        _check(lib().pw_step_to(self.h, _ptr(u, g, "u"), _ptr(v, g, "v"), _ptr(w, g, "w"), _ptr(nu, g, "nu"),
                                _ptr(nv, g, "nv"), _ptr(nw, g, "nw"), float(dt), sp[0] if sp else None,
                                _stream_ptr(stream)), "pw_step_to")

    def adjoint(self, u, v, w, lsu, lsv, lsw, gu, gv, gw, alpha=1.0, flags=0, stream=None):
        """g = [g | l | 0] + alpha * J(u,v,w)^T l (see pw_adjoint for flags)."""
        g = self.grid
        _check(lib().pw_adjoint(self.h, _ptr(u, g, "u"), _ptr(v, g, "v"), _ptr(w, g, "w"), _ptr(lsu, g, "lsu"),
                                _ptr(lsv, g, "lsv"), _ptr(lsw, g, "lsw"), _ptr(gu, g, "gu"), _ptr(gv, g, "gv"),
                                _ptr(gw, g, "gw"), float(alpha), int(flags), _stream_ptr(stream)), "pw_adjoint")

    def fill_halo_periodic(self, f, stream=None):
        _check(lib().pw_fill_halo_periodic(self.h, _ptr(f, self.grid, "f"), _stream_ptr(stream)),
               "pw_fill_halo_periodic")

    def error_norms(self, test, ref, k0=1, k1=None, scale=1.0, stream=None):
        """(max|t-r|, max|r|, sum (t-r)^2, sum r^2) over levels k0..k1; ref is a
        dense (nz+2, ny+2, nx+2) float64 tensor (moved to the device)."""
        g = self.grid
        k1 = g.nz if k1 is None else k1
        r = torch.as_tensor(ref, dtype=torch.float64).to(device=test.device).contiguous()
        if tuple(r.shape) != (g.nz + 2, g.ny + 2, g.nx + 2):
            raise ValueError("ref must have shape (nz+2, ny+2, nx+2)")
        out = (ctypes.c_double * 4)()
        _check(lib().pw_error_norms(self.h, _ptr(test, g, "test"), float(scale), ctypes.c_void_p(r.data_ptr()),
                                    int(k0), int(k1), ctypes.cast(out, _dp), _stream_ptr(stream)),
               "pw_error_norms")
        return np.array(out[:])

    def weighted_dot(self, a, b, wk=None, k0=1, k1=None, sa=1.0, sb=1.0, stream=None):
        g = self.grid
        k1 = g.nz if k1 is None else k1
        wp = None
        if wk is not None:
            wk = np.ascontiguousarray(wk, dtype=np.float64)
            if wk.shape != (g.nz + 2,):
                raise ValueError("wk must have nz+2 entries")
            wp = wk.ctypes.data_as(_dp)
        out = ctypes.c_double()
        _check(lib().pw_weighted_dot(self.h, _ptr(a, g, "a"), float(sa), _ptr(b, g, "b"), float(sb), wp,
                                     int(k0), int(k1), ctypes.byref(out), _stream_ptr(stream)), "pw_weighted_dot")
        return float(out.value)

    def selftest_wait_timeout(self, limit_ns=100_000_000, stream=None):
        _check(lib().pw_selftest_wait_timeout(self.h, int(limit_ns), _stream_ptr(stream)),
               "pw_selftest_wait_timeout")

    def weighted_dot_noalloc(self, a, b, wk=None, k0=1, k1=None, sa=1.0, sb=1.0, stream=None):
        """weighted_dot with its scratch in the library's static device array:
        no device allocation at call time (see pw_weighted_dot_noalloc)."""
        g = self.grid
        k1 = g.nz if k1 is None else k1
        wp = None
        if wk is not None:
            wk = np.ascontiguousarray(wk, dtype=np.float64)
            if wk.shape != (g.nz + 2,):
                raise ValueError("wk must have nz+2 entries")
            wp = wk.ctypes.data_as(_dp)
        out = ctypes.c_double()
        _check(lib().pw_weighted_dot_noalloc(self.h, _ptr(a, g, "a"), float(sa), _ptr(b, g, "b"), float(sb), wp,
                                             int(k0), int(k1), ctypes.byref(out), _stream_ptr(stream)),
               "pw_weighted_dot_noalloc")
        return float(out.value)

    def sync(self, stream=None):
        _check(lib().pw_sync(self.h, _stream_ptr(stream)), "pw_sync")


class Batch:
    """A pw_batch_t: independent grids (one dtype) in one persistent,
    graph-replayed launch."""

    def __init__(self, grids, coeffs_list):
        if len(grids) != len(coeffs_list) or not grids:
            raise ValueError("need one coefficient set per grid")
        self.grids = list(grids)
        n = len(grids)
        self._keep = []
        cs = (pw_coeffs_t * n)()
        for q, (g, c) in enumerate(zip(grids, coeffs_list)):
            arrs = [np.ascontiguousarray(getattr(c, a) if not isinstance(c, dict) else c[a], dtype=np.float64)
                    for a in ("tzc1", "tzc2", "tzd1", "tzd2")]
            self._keep.append(arrs)
            get = (lambda k: c[k]) if isinstance(c, dict) else (lambda k: getattr(c, k))
            cs[q] = pw_coeffs_t(float(get("tcx")), float(get("tcy")), *[a.ctypes.data_as(_dp) for a in arrs])
        gs = (pw_grid_t * n)(*[g.c for g in grids])
        h = ctypes.c_void_p()
        _check(lib().pw_batch_create(n, gs, cs, ctypes.byref(h)), "pw_batch_create")
        self.h = h
        self._keep = None

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().pw_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_config(self, lanes_x=0, ty=0, stages=0, ctas_per_sm=0, rows=0, cells=0):
        """Tile shape of the batched kernel (0 = default field); rows = rows
        per thread (2: packed FP32x2 on row pairs; 3: one row, its cells
        packed as FP32x2 pairs along x; both 16-bit storage); cells = cells
        per thread along x (4, or 8 with x pairs when every nx allows)."""
        _check(lib().pw_batch_set_config(self.h, int(lanes_x), int(cells), int(ty), int(stages), int(ctas_per_sm),
                                         int(rows)), "pw_batch_set_config")

    def set_narrow_columns(self, enable=True):
        """March a grid's last column with tiles half as wide when it holds at
        most half a tile (shapes with a narrow partner only; on by default)."""
        _check(lib().pw_batch_set_narrow_columns(self.h, 1 if enable else 0), "pw_batch_set_narrow_columns")

    def narrow_shape(self):
        """The narrow shape in use, {"lanes_x", "cells", "ty"} (zeros: none)."""
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().pw_batch_narrow_shape(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "pw_batch_narrow_shape")
        return {"lanes_x": a.value, "cells": b.value, "ty": c.value}

    def info(self):
        ni, cells, ctas = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(lib().pw_batch_info(self.h, ctypes.byref(ni), ctypes.byref(cells), ctypes.byref(ctas)),
               "pw_batch_info")
        return {"items": ni.value, "cells": cells.value, "ctas": ctas.value}

    def tendencies(self, us, vs, ws, sus, svs, sws, scale=None, stream=None):
        n = len(self.grids)
        tabs = []
        for name, lst in (("u", us), ("v", vs), ("w", ws), ("su", sus), ("sv", svs), ("sw", sws)):
            if len(lst) != n:
                raise ValueError(f"{name}: need {n} tensors")
            tabs.append((_VP * n)(*[_ptr(t, g, name).value for t, g in zip(lst, self.grids)]))
        sp = _scale_arg(scale)
        _check(lib().pw_batch_tendencies(self.h, *tabs, sp[0] if sp else None, _stream_ptr(stream)),
               "pw_batch_tendencies")

    def sync(self, stream=None):
        _check(lib().pw_batch_sync(self.h, _stream_ptr(stream)), "pw_batch_sync")
