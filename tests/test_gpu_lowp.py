"""BF16 / FP16 storage of u, v, w and su, sv, sw with FP32 arithmetic, through
the C ABI, against the FP64 oracle.

Two per-cell bounds, with A(q) the oracle's magnitude sum of the terms
(oracle.abs_terms) and u_s the storage format's unit roundoff:
  kernel:  |gpu - s64(q~)| <= u_s |s64(q~)| + 2^-19 A(q~) + floor
           (q~ = the dequantised stored inputs: only output rounding and FP32
           arithmetic separate the two);
  total:   |gpu - s64(q)|  <= u_s |s64(q)| + (2 u_s + 2^-19) A(q) + floor
           (q = the original FP32 fields: adds the effect of rounding every
           input once; the factor 1.05 on A covers the second-order terms).
floor covers outputs that land in the format's subnormal range.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2301_13016_gb300 as pwlib
from paper_2301_13016_gb300 import inputs, precision
from gpu_util import NAN, interior

pytestmark = pytest.mark.gpu


def _run_lowp(nx, ny, nz, dtype, smooth, kernel=0):
    c = inputs.make_coeffs(nz)
    f = inputs.smooth_fields(nx, ny, nz) if smooth else inputs.random_fields(nx, ny, nz)
    maxabs = [float(x.abs().max()) for x in f]
    sc = precision.suggest_scales(maxabs, c, dtype)
    g = pwlib.Grid(nx, ny, nz, dtype=dtype)
    h = pwlib.PW(g, c)
    h.set_kernel(kernel)
    dev = [g.from_dense(x, scale=s) for x, s in zip(f, sc[:3])]
    outs = [g.alloc(fill=NAN) for _ in range(3)]
    h.tendencies(*dev, *outs, scale=sc)
    h.sync()
    got = [g.to_dense(o).numpy() / s for o, s in zip(outs, sc[3:])]
    q_tilde = [g.to_dense(d, s).numpy() for d, s in zip(dev, sc[:3])]
    q = [x.numpy().astype(np.float64) for x in f]
    return c, sc, q, q_tilde, got, h


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("smooth", [False, True], ids=["random", "smooth"])
@pytest.mark.parametrize("shape", [(128, 24, 16), (388, 13, 6)], ids=["128x24x16", "388x13x6"])
def test_lowp_storage_bounds(dtype, smooth, shape):
    c, sc, q, qt, got, h = _run_lowp(*shape, dtype, smooth)
    assert h.last_kernel == 2
    us = precision.UNIT_ROUNDOFF[dtype]
    # kernel bound: oracle on the dequantised stored inputs
    ref_t = oracle.tendencies(*qt, c)
    a_t = oracle.abs_terms(*qt, c)
    for x, r, a, so in zip(got, ref_t, a_t, sc[3:]):
        floor = 2 * precision.MIN_NORMAL[dtype] / so
        err = np.abs(interior(x) - interior(r))
        assert np.all(err <= us * np.abs(interior(r)) + 2.0 ** -19 * interior(a) + floor)
    # total bound: oracle on the original FP32 fields
    ref = oracle.tendencies(*q, c)
    a_q = oracle.abs_terms(*q, c)
    for x, r, a, so in zip(got, ref, a_q, sc[3:]):
        floor = 2 * precision.MIN_NORMAL[dtype] / so
        err = np.abs(interior(x) - interior(r))
        assert np.all(err <= us * np.abs(interior(r)) + (2 * us + 2.0 ** -19) * interior(a) * 1.05 + floor)


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_lowp_generic_kernel_and_agreement(dtype):
    c, sc, q, qt, a, h1 = _run_lowp(128, 16, 10, dtype, False, kernel=1)
    assert h1.last_kernel == 1
    c, sc, q, qt, b, h2 = _run_lowp(128, 16, 10, dtype, False, kernel=2)
    assert h2.last_kernel == 2
    us = precision.UNIT_ROUNDOFF[dtype]
    ref_t = oracle.tendencies(*qt, c)
    a_t = oracle.abs_terms(*qt, c)
    for x, y, r, at, so in zip(a, b, ref_t, a_t, sc[3:]):
        floor = 2 * precision.MIN_NORMAL[dtype] / so
        # the generic kernel meets the same per-cell kernel bound
        assert np.all(np.abs(interior(x) - interior(r)) <= us * np.abs(interior(r)) + 2.0 ** -19 * interior(at) + floor)
        # the two kernels round FP32 results evaluated in different orders:
        # one storage unit each plus both arithmetic errors apart
        assert np.all(np.abs(interior(x) - interior(y)) <=
                      2 * us * np.abs(interior(r)) + 2.0 ** -18 * interior(at) + 2 * floor)


def test_normwise_errors_within_stated_bounds():
    """The normwise errors max|err|/max|ref| against the FP64 oracle on the
    FP32 fields stay inside the stated bounds: BF16 1e-2 (random) / 1e-1
    (smooth), FP16 2e-3 / 1e-2."""
    stated = {("bf16", False): 1e-2, ("bf16", True): 1e-1, ("f16", False): 2e-3, ("f16", True): 1e-2}
    for (dtype, smooth), bound in stated.items():
        c, sc, q, qt, got, _ = _run_lowp(256, 32, 16, dtype, smooth)
        ref = oracle.tendencies(*q, c)
        for x, r in zip(got, ref):
            rel = np.abs(interior(x) - interior(r)).max() / np.abs(interior(r)).max()
            assert rel <= bound, (dtype, smooth, rel)


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("ty,nseg", [(4, 1), (8, 3)])
def test_eight_cells_per_thread(dtype, ty, nseg):
    """16-bit storage with 8 cells per thread (one 16-byte access per row
    vector): the kernel bound on a ragged tile (264 = 2 x 128 + 8 columns),
    and agreement with the 4-cell kernel to one storage unit."""
    nx, ny, nz = 264, 13, 10
    c = inputs.make_coeffs(nz)
    f = inputs.random_fields(nx, ny, nz)
    sc = precision.suggest_scales([float(x.abs().max()) for x in f], c, dtype)
    g = pwlib.Grid(nx, ny, nz, dtype=dtype)
    h = pwlib.PW(g, c)
    dev = [g.from_dense(x, scale=s) for x, s in zip(f, sc[:3])]
    res = {}
    for cells in (4, 8):
        h.set_tma_config(ty, 4, nseg, lanes_x=16, cells=cells)
        outs = [g.alloc(fill=NAN) for _ in range(3)]
        h.tendencies(*dev, *outs, scale=sc)
        h.sync()
        assert h.last_kernel == 2
        res[cells] = [g.to_dense(o).numpy() / s for o, s in zip(outs, sc[3:])]
    qt = [g.to_dense(d, s).numpy() for d, s in zip(dev, sc[:3])]
    ref = oracle.tendencies(*qt, c)
    a = oracle.abs_terms(*qt, c)
    us = precision.UNIT_ROUNDOFF[dtype]
    for x, y, r, at, so in zip(res[8], res[4], ref, a, sc[3:]):
        floor = 2 * precision.MIN_NORMAL[dtype] / so
        assert np.all(np.abs(interior(x) - interior(r)) <= us * np.abs(interior(r)) + 2.0 ** -19 * interior(at) + floor)
        assert np.all(np.abs(interior(x) - interior(y)) <= 2 * us * np.abs(interior(r)) + 2.0 ** -18 * interior(at) + 2 * floor)
    # nx = 132 = 4 mod 8: source terms with 8 cells per thread (the row's last
    # vector stores 4 cells) equal the 4-cell kernel's bits; fused steps need
    # nx to be a multiple of 8
    g2 = pwlib.Grid(132, 8, 4, dtype=dtype)
    f2 = inputs.random_fields(132, 8, 4)
    h2 = pwlib.PW(g2, inputs.make_coeffs(4))
    d2 = [g2.from_dense(x, scale=s) for x, s in zip(f2, sc[:3])]
    got = {}
    for cells in (4, 8):
        h2.set_tma_config(4, 4, 0, lanes_x=16, cells=cells)
        o2 = [g2.alloc(fill=NAN) for _ in range(3)]
        h2.tendencies(*d2, *o2, scale=sc)
        h2.sync()
        got[cells] = [t.view(torch.int16).clone() for t in o2]
    for a_, b_ in zip(got[4], got[8]):
        assert torch.equal(a_, b_)
    with pytest.raises(pwlib.PwError) as e:
        h2.step(*d2, *[g2.alloc() for _ in range(3)], 1.0, 1, scale=sc[:3])
    assert e.value.status == pwlib.PW_ERR_UNSUPPORTED


# (lanes, rows, stages, cells, form): form 2 = two rows per thread (each cell
# paired with the cell below it), 3 = one row per thread with its cells paired
# along x (cell q with cell q + cells/2)
PAIRED = [(32, 8, 4, 4, 2), (32, 16, 4, 4, 2), (16, 8, 4, 4, 2),
          (16, 4, 4, 8, 3), (16, 8, 4, 8, 3), (16, 16, 4, 8, 3), (32, 4, 4, 4, 3), (32, 8, 4, 4, 3),
          (16, 8, 4, 4, 3), (8, 8, 4, 8, 3), (8, 16, 4, 8, 3)]


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("cfg", PAIRED, ids=["x".join(map(str, p)) for p in PAIRED])
def test_two_rows_per_thread_bitwise(dtype, cfg):
    """The packed FP32x2 forms (two rows per thread, or the cells of one row
    paired along x) give the same bits as one scalar row per thread, for the
    source terms and for fused steps, on tiles ragged in x (264 = 2 x 128 + 8
    columns) and in y (13 rows: the last row pair has its second row outside
    the grid)."""
    nx, ny, nz = 264, 13, 10
    c = inputs.make_coeffs(nz)
    f = inputs.random_fields(nx, ny, nz)
    sc = precision.suggest_scales([float(x.abs().max()) for x in f], c, dtype)
    g = pwlib.Grid(nx, ny, nz, dtype=dtype)
    lx, ty, st, cells, rows = cfg
    res = {}
    for key, shape in (("one", (32, 4, 4, 4, 1)), ("two", cfg)):
        h = pwlib.PW(g, c)
        h.set_tma_config(shape[1], shape[2], 0, lanes_x=shape[0], cells=shape[3], rows=shape[4])
        dev = [g.from_dense(x, scale=s) for x, s in zip(f, sc[:3])]
        outs = [g.alloc(fill=NAN) for _ in range(3)]
        h.tendencies(*dev, *outs, scale=sc)
        tmp = [g.alloc(fill=NAN) for _ in range(3)]
        h.step(*dev, *tmp, 0.5, 3, scale=sc[:3])
        h.sync()
        assert h.last_kernel == 2
        res[key] = [g.view(t).contiguous().view(torch.int16) for t in outs + dev]
    for a, b in zip(res["one"], res["two"]):
        assert torch.equal(a, b)


def test_two_rows_per_thread_needs_16bit_storage():
    g = pwlib.Grid(128, 8, 4)
    with pytest.raises(pwlib.PwError) as e:
        pwlib.PW(g, inputs.make_coeffs(4)).set_tma_config(8, 4, 0, lanes_x=32, cells=4, rows=2)
    assert e.value.status == pwlib.PW_ERR_UNSUPPORTED


def test_automatic_launch_shapes():
    """The automatic k-march shape per call: FP32 32 lanes x 4 cells x 4 rows;
    16-bit source terms 16 x 8 x 8 with the cells paired along x (rows = 3);
    16-bit steps the same when nx is a multiple of 8, else 32 x 4 x 4 in x
    pairs; 16 x 4 x 4 for grids at most 64 columns wide, with k segments of
    2 levels; a shape set by pw_set_tma_config is used as given (zero fields
    at the scalar defaults) for every call."""
    c = inputs.make_coeffs(8)

    def pick(g, step=False):
        return {k: v for k, v in pwlib.PW(g, c).tma_config(step).items() if k != "nseg"}

    f32 = dict(lanes_x=32, cells=4, ty=4, stages=4, rows=1)
    for step in (False, True):
        assert pick(pwlib.Grid(256, 64, 8), step) == f32
    for dtype in ("bf16", "f16"):
        xp8 = dict(lanes_x=16, cells=8, ty=8, stages=4, rows=3)
        for nx in (256, 260):
            assert pick(pwlib.Grid(nx, 64, 8, dtype=dtype)) == xp8
        assert pick(pwlib.Grid(256, 64, 8, dtype=dtype), True) == xp8
        assert pick(pwlib.Grid(260, 64, 8, dtype=dtype), True) == dict(f32, rows=3)
    for dtype in ("f32", "bf16"):
        for step in (False, True):
            assert pwlib.PW(pwlib.Grid(64, 64, 8, dtype=dtype), c).tma_config(step) == dict(
                lanes_x=16, cells=4, ty=4, stages=4, nseg=4, rows=1)
    h = pwlib.PW(pwlib.Grid(256, 64, 8, dtype="bf16"), c)
    h.set_tma_config(8, 4, 2, lanes_x=32, cells=4, rows=2)
    for step in (False, True):
        assert h.tma_config(step) == dict(lanes_x=32, cells=4, ty=8, stages=4, nseg=2, rows=2)
    h.set_tma_config(ty=8)
    assert h.tma_config() == dict(f32, ty=8, nseg=h.tma_config()["nseg"])
    h.set_tma_config()
    assert pick(pwlib.Grid(256, 64, 8, dtype="bf16")) == {k: v for k, v in h.tma_config().items() if k != "nseg"}


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_host_path_16bit_matches_device_path(dtype):
    """pw_tendencies_host with 16-bit storage (the packed two-row shape,
    pipelined in 4-level chunks; FP16 with scales) gives the device path's
    bits."""
    nx, ny, nz = 256, 20, 64
    c = inputs.make_coeffs(nz)
    f = inputs.random_fields(nx, ny, nz)
    sc = precision.suggest_scales([float(x.abs().max()) for x in f], c, dtype)
    g = pwlib.Grid(nx, ny, nz, dtype=dtype)
    h = pwlib.PW(g, c)
    dev = [g.from_dense(x, scale=s) for x, s in zip(f, sc[:3])]
    outs = [g.alloc(fill=NAN) for _ in range(3)]
    h.tendencies(*dev, *outs, scale=sc)
    h.sync()
    hin = [t.cpu().pin_memory() for t in dev]
    hout = [torch.zeros(g.alloc_elems, dtype=g.torch_dtype).pin_memory() for _ in range(3)]
    h.tendencies_host(*hin, *hout, scale=sc)
    assert h.last_kernel == 2
    for o, t in zip(outs, hout):
        a = g.view(o)[1:-1, 1:-1, 1:-1].contiguous().view(torch.int16).cpu()
        b = g.view(t)[1:-1, 1:-1, 1:-1].contiguous().view(torch.int16)
        assert torch.equal(a, b)
