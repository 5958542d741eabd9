"""Plant plausible mistakes in copies of the CPU oracle and check that the pins
in tests/pins.py catch every one (no GPU; the mistakes are planted on the CPU,
in temporary copies of oracle/pw_oracle_body.h, never in the repository).

Each mutant is a one-line edit of the kind a transcription slip makes: a
wrong neighbour index, a dropped term, a flipped sign, a swapped coefficient,
a transposed operand, the lid or surface level mishandled.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import pins

ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")

# (name, old text, new text, occurrence of old text to replace: 0 = first)
MUTANTS = [
    ("su_pair_sum_x_index", "REAL ax_w = u[IDX(k, j, i)] + u[IDX(k, j, i - 1)];",
     "REAL ax_w = u[IDX(k, j, i)] + u[IDX(k, j, i + 1)];", 0),
    ("su_pair_sum_y_index", "REAL ay_s = v[IDX(k, j - 1, i)] + v[IDX(k, j - 1, i + 1)];",
     "REAL ay_s = v[IDX(k, j - 1, i)] + v[IDX(k, j - 1, i - 1)];", 0),
    ("su_neighbour_y_index", "REAL py_n = u[IDX(k, j + 1, i)] * ay_n;",
     "REAL py_n = u[IDX(k, j - 1, i)] * ay_n;", 0),
    ("su_neighbour_z_index", "REAL pz_b = u[IDX(k - 1, j, i)] * az_b;",
     "REAL pz_b = u[IDX(k, j, i)] * az_b;", 0),
    ("su_top_w_average", "REAL az_t = w[IDX(k, j, i)] + w[IDX(k, j, i + 1)];",
     "REAL az_t = w[IDX(k, j, i)] + w[IDX(k, j, i - 1)];", 0),
    ("su_z_sign", "tzc1[k] * pz_b - tzc2[k] * pz_t : tzc1[k] * pz_b;",
     "tzc1[k] * pz_b + tzc2[k] * pz_t : tzc1[k] * pz_b;", 0),
    ("su_drop_x_term", "su[c] = tx + ty + tz;", "su[c] = ty + tz;", 0),
    ("su_tcx_for_tcy", "REAL tx = tcx * (px_w - px_e);", "REAL tx = tcy * (px_w - px_e);", 0),
    ("su_lid_flux_kept", "REAL tz = (k < nz) ? tzc1[k] * pz_b - tzc2[k] * pz_t : tzc1[k] * pz_b;",
     "REAL tz = tzc1[k] * pz_b - tzc2[k] * u[IDX(k + 1, j, i)] * az_t;", 0),
    ("sv_u_average_index", "u[IDX(k, j + 1, i - 1)]", "u[IDX(k, j - 1, i - 1)]", 0),
    ("sv_w_average_index", "w[IDX(k - 1, j + 1, i)]", "w[IDX(k - 1, j, i + 1)]", 0),
    ("sv_pair_sum_y_index", "REAL ay_s = v[IDX(k, j, i)] + v[IDX(k, j - 1, i)];",
     "REAL ay_s = v[IDX(k, j, i)] + v[IDX(k, j + 1, i)];", 0),
    ("sv_neighbour_x_index", "REAL px_e = v[IDX(k, j, i + 1)] * ax_e;",
     "REAL px_e = v[IDX(k, j, i)] * ax_e;", 0),
    ("sv_y_sign", "REAL ty = tcy * (py_s - py_n);", "REAL ty = tcy * (py_n - py_s);", 1),
    ("sw_v_average_level", "REAL ay_n = v[IDX(k, j, i)] + v[IDX(k + 1, j, i)];",
     "REAL ay_n = v[IDX(k, j, i)] + v[IDX(k - 1, j, i)];", 0),
    ("sw_tzd2_for_tzd1", "REAL tz = tzd1[k] * pz_b - tzd2[k] * pz_t;",
     "REAL tz = tzd1[k] * pz_b - tzd1[k] * pz_t;", 0),
    ("sw_neighbour_z_index", "REAL pz_t = w[IDX(k + 1, j, i)] * az_t;",
     "REAL pz_t = w[IDX(k, j, i)] * az_t;", 0),
    ("sw_transposed_operand", "REAL px_w = w[IDX(k, j, i - 1)] * ax_w;",
     "REAL px_w = u[IDX(k, j, i - 1)] * ax_w;", 0),
    ("surface_level_computed", "if (k == 1) {", "if (k == 0) {", 0),
    ("sw_x_average_level", "REAL ax_e = u[IDX(k, j, i)] + u[IDX(k + 1, j, i)];",
     "REAL ax_e = u[IDX(k, j, i)] + u[IDX(k - 1, j, i)];", 0),
]


def _replace_nth(text, old, new, n):
    pos = -1
    for _ in range(n + 1):
        pos = text.find(old, pos + 1)
        if pos < 0:
            raise ValueError(f"occurrence {n} of {old!r} not found")
    return text[:pos] + new + text[pos + len(old):]


def _build_variant(tmpdir, body_text):
    shutil.copy(os.path.join(ORACLE_DIR, "pw_oracle.c"), tmpdir)
    with open(os.path.join(tmpdir, "pw_oracle_body.h"), "w") as fh:
        fh.write(body_text)
    lib = os.path.join(tmpdir, "libvariant.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", lib,
                    os.path.join(tmpdir, "pw_oracle.c")], check=True)
    return lib


def _tend_from(lib_path):
    lib = ctypes.CDLL(lib_path)
    dp = ctypes.POINTER(ctypes.c_double)
    fn = lib.pw_oracle_tendencies_f64
    fn.argtypes = [ctypes.c_int] * 3 + [dp] * 3 + [ctypes.c_double] * 2 + [dp] * 7
    fn.restype = None

    def tend(u, v, w, c):
        u, v, w = (np.ascontiguousarray(a, dtype=np.float64) for a in (u, v, w))
        nz, ny, nx = (s - 2 for s in u.shape)
        tz = [np.ascontiguousarray(getattr(c, n), dtype=np.float64) for n in ("tzc1", "tzc2", "tzd1", "tzd2")]
        out = [np.zeros_like(u) for _ in range(3)]
        p = lambda a: a.ctypes.data_as(dp)
        fn(nx, ny, nz, p(u), p(v), p(w), float(c.tcx), float(c.tcy), *[p(t) for t in tz], *[p(o) for o in out])
        return tuple(out)
    return tend


@pytest.fixture(scope="module")
def body():
    with open(os.path.join(ORACLE_DIR, "pw_oracle_body.h")) as fh:
        return fh.read()


def test_unmutated_copy_passes(tmp_path, body):
    tend = _tend_from(_build_variant(str(tmp_path), body))
    assert pins.failures(tend) == []


@pytest.mark.parametrize("name,old,new,occ", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, body, name, old, new, occ):
    text = _replace_nth(body, old, new, occ)
    assert text != body
    tend = _tend_from(_build_variant(str(tmp_path), text))
    caught = pins.failures(tend)
    assert caught, f"mutant {name} passed every pin"
