"""The C ABI without a GPU: libpw.so loads, exports every entry point that
include/pw.h declares, and rejects bad arguments on the host before any CUDA
call.  (The library is built by __graft_entry__.build(); nvcc cross-compiles.)
"""
import ctypes
import os
import re

import pytest

import paper_2301_13016_gb300 as pwlib
from paper_2301_13016_gb300 import pw as pwmod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pw.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(pw_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(pwmod.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return pwlib.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pw_create", "pw_tendencies", "pw_destroy", "pw_fill_halo_periodic", "pw_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(L):
    for name in declared_functions():
        assert hasattr(L, name), f"{name} declared in pw.h but not exported by libpw.so"


def test_binding_covers_every_declared_symbol():
    bound = {n for n, _, _ in pwmod.SIGNATURES}
    assert set(declared_functions()) == bound


def test_no_torch_or_cuda_types_in_header():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)   # code, not comments
    for bad in ("torch", "at::", "c10", "cudaStream_t", "#include <cuda"):
        assert bad not in text


def test_grid_default_layout(L):
    for dtype, es in (("f32", 4), ("bf16", 2), ("f16", 2)):
        for (nx, ny, nz, halo) in ((64, 64, 64, 1), (2048, 2048, 64, 1), (36, 12, 5, 1), (40, 16, 8, 3)):
            g = pwlib.Grid(nx, ny, nz, halo=halo, dtype=dtype)
            assert g.pitch_j >= nx + 2 * halo and (g.pitch_j * es) % 128 == 0
            assert g.pitch_k == g.pitch_j * (ny + 2 * halo)
            # interior row start (i = 1) on a 128-byte boundary
            assert ((g.origin + 1) * es) % 128 == 0 or halo > 1
            # the last element fits the allocation
            last = g.origin + (nz + 1) * g.pitch_k + (ny + halo) * g.pitch_j + nx + halo
            assert last < g.alloc_elems
            # the most negative element (k=0, j=1-halo, i=1-halo) is in range
            assert g.origin + (1 - halo) * g.pitch_j + (1 - halo) >= 0




def test_create_rejects_bad_grids_on_host(L):
    tz = (ctypes.c_double * 10)()
    dp = ctypes.POINTER(ctypes.c_double)
    c = pwmod.pw_coeffs_t(0.0025, 0.0025, ctypes.cast(tz, dp), ctypes.cast(tz, dp), ctypes.cast(tz, dp),
                          ctypes.cast(tz, dp))
    h = ctypes.c_void_p()
    bad = [
        pwmod.pw_grid_t(8, 8, 2, 1, 10, 100, 0, 0),      # nz < 3
        pwmod.pw_grid_t(0, 8, 8, 1, 10, 100, 0, 0),      # nx < 1
        pwmod.pw_grid_t(8, 8, 8, 1, 9, 100, 0, 0),       # pitch_j < nx + 2
        pwmod.pw_grid_t(8, 8, 8, 1, 10, 99, 0, 0),       # pitch_k < pitch_j*(ny+2)
        pwmod.pw_grid_t(8, 8, 8, 0, 10, 100, 0, 0),      # halo < 1
        pwmod.pw_grid_t(8, 8, 8, 2, 12, 144, 0, 0),      # origin leaves no room for halo 2
        pwmod.pw_grid_t(8, 8, 8, 1, 10, 100, 0, 7),      # unknown dtype
    ]
    for g in bad:
        st = L.pw_create(ctypes.byref(g), ctypes.byref(c), ctypes.byref(h))
        assert st == pwlib.PW_ERR_ARG, (g.nx, g.nz, st)
        assert h.value is None
        assert L.pw_last_error()
    good = pwmod.pw_grid_t(8, 8, 8, 1, 10, 100, 0, 0)
    assert L.pw_create(ctypes.byref(good), None, ctypes.byref(h)) == pwlib.PW_ERR_ARG
    assert L.pw_create(None, ctypes.byref(c), ctypes.byref(h)) == pwlib.PW_ERR_ARG


def test_null_handle_is_rejected(L):
    assert L.pw_tendencies(None, None, None, None, None, None, None, None, None) == pwlib.PW_ERR_ARG
    assert L.pw_fill_halo_periodic(None, None, None) == pwlib.PW_ERR_ARG
    assert L.pw_sync(None, None) == pwlib.PW_ERR_ARG
    assert L.pw_destroy(None) == pwlib.PW_OK
    assert L.pw_status_string(pwlib.PW_ERR_DEVICE_TIMEOUT) == b"PW_ERR_DEVICE_TIMEOUT"
    # the batch's host-side entry points check their handle before any CUDA call
    assert L.pw_batch_set_narrow_columns(None, 1) == pwlib.PW_ERR_ARG
    assert L.pw_batch_narrow_shape(None, None, None, None) == pwlib.PW_ERR_ARG
    assert L.pw_batch_set_config(None, 16, 4, 16, 4, 0, 1) == pwlib.PW_ERR_ARG
    assert L.pw_batch_info(None, None, None, None) == pwlib.PW_ERR_ARG
    assert L.pw_batch_destroy(None) == pwlib.PW_OK


def test_failure_injection_arguments(L):
    """pw_inject_failures takes kind 0 (allocations) or 1 (descriptor
    encodings) and a count >= 0; count 0 clears (no GPU needed)."""
    assert L.pw_inject_failures(2, 1) == pwlib.PW_ERR_ARG
    assert L.pw_inject_failures(-1, 1) == pwlib.PW_ERR_ARG
    assert L.pw_inject_failures(0, -1) == pwlib.PW_ERR_ARG
    for kind in (0, 1):
        assert L.pw_inject_failures(kind, 3) == pwlib.PW_OK
        assert L.pw_inject_failures(kind, 0) == pwlib.PW_OK


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(pwmod, "_LIB", None)
    monkeypatch.setattr(pwmod, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        pwmod.lib()


def test_debug_layout_check_matches_the_layout(L):
    """The rule the debug bounds build applies to every store, on the host:
    cells of levels 1..nz, interior (or interior plus lateral halo), never
    row padding or the z-halo planes."""
    g = pwmod.pw_grid_t()
    n_elems = ctypes.c_int64()
    assert L.pw_grid_default(100, 7, 5, 1, 0, ctypes.byref(g), ctypes.byref(n_elems)) == pwlib.PW_OK
    off = lambda k, j, i: g.origin + k * g.pitch_k + j * g.pitch_j + i
    chk = lambda o, n, inner: L.pw_debug_layout_check(ctypes.byref(g), o, n, inner)
    assert g.pitch_j > g.nx + 2                          # the default layout pads its rows
    for k in (1, 3, 5):
        assert chk(off(k, 1, 1), 4, 1) == 1               # an interior vector
        assert chk(off(k, 7, 97), 4, 1) == 1              # the row's last one
        assert chk(off(k, 7, 98), 4, 1) == 0              # one cell past the interior
        assert chk(off(k, 7, 98), 4, 0) == 1              # ... which the halo allows
        assert chk(off(k, 7, 98), 5, 0) == 0              # ... but not into the padding
        assert chk(off(k, 0, 0), 1, 0) == 1 and chk(off(k, 0, 0), 1, 1) == 0   # a halo corner
        assert chk(off(k, 8, 101), 1, 0) == 1              # the top halo row's last cell
        assert chk(off(k, 3, 102), 1, 0) == 0            # row padding
    assert chk(off(0, 1, 1), 1, 0) == 0 and chk(off(6, 1, 1), 1, 0) == 0   # z-halo planes
    assert chk(off(1, 1, 1) - 10 ** 6, 1, 0) == 0 and chk(off(1, 1, 1), 0, 0) == -1
    g2 = pwmod.pw_grid_t()
    assert L.pw_grid_default(64, 9, 4, 2, 1, ctypes.byref(g2), ctypes.byref(n_elems)) == pwlib.PW_OK
    off2 = lambda k, j, i: g2.origin + k * g2.pitch_k + j * g2.pitch_j + i
    assert L.pw_debug_layout_check(ctypes.byref(g2), off2(2, -1, -1), 1, 0) == 1   # halo 2 corner
    assert L.pw_debug_layout_check(ctypes.byref(g2), off2(2, 11, 66), 1, 0) == 1
    assert L.pw_debug_layout_check(ctypes.byref(g2), off2(2, 5, 67), 1, 0) == 0   # row padding
    # a layout with a padding row between levels: that row is never writable
    g3 = pwmod.pw_grid_t(100, 7, 5, 1, 160, 160 * 10, 31, 0)
    off3 = lambda k, j, i: g3.origin + k * g3.pitch_k + j * g3.pitch_j + i
    assert L.pw_debug_layout_check(ctypes.byref(g3), off3(3, 8, 1), 1, 0) == 1
    assert L.pw_debug_layout_check(ctypes.byref(g3), off3(3, 9, 1), 1, 0) == 0
    assert L.pw_debug_bounds_build() in (0, 1)
