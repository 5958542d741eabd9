"""Batched form through the C ABI: many independent grids of uneven sizes in
one persistent, graph-replayed launch.  Each grid's result is checked against
the FP64 oracle and against the single-grid k-march kernel of the same tile
shape (same per-cell arithmetic: bit-identical)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2301_13016_gb300 as pwlib
from paper_2301_13016_gb300 import autotune, inputs
from gpu_util import NAN, interior

pytestmark = pytest.mark.gpu


def _make_batch(shapes, dtype="f32", seed0=10):
    grids, coeffs, fields, dev = [], [], [], []
    for q, (nx, ny, nz) in enumerate(shapes):
        g = pwlib.Grid(nx, ny, nz, dtype=dtype)
        # every other grid with the anelastic coefficient set (tzc1 != tzc2)
        c = inputs.make_coeffs(nz, dx=100.0 + q, dy=90.0 + q, anelastic=(q % 2 == 1))
        f = inputs.random_fields(nx, ny, nz, seeds=(seed0 + 3 * q, seed0 + 3 * q + 1, seed0 + 3 * q + 2))
        grids.append(g)
        coeffs.append(c)
        fields.append(f)
        dev.append([g.from_dense(x) for x in f])
    b = pwlib.Batch(grids, coeffs)
    outs = [[g.alloc(fill=NAN) for _ in range(3)] for g in grids]
    return b, grids, coeffs, fields, dev, outs


def _run(b, dev, outs, scale=None):
    b.tendencies([d[0] for d in dev], [d[1] for d in dev], [d[2] for d in dev],
                 [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs], scale=scale)
    b.sync()


SHAPES = [(32, 40, 8), (384, 36, 5), (100, 17, 12), (64, 64, 3), (260, 9, 20), (36, 300, 6), (128, 4, 4)]


@pytest.mark.parametrize("cfg", [(32, 4, 4), (32, 8, 4), (16, 4, 4), (16, 8, 4), (16, 16, 4), (8, 16, 4), (32, 16, 4)])
def test_batch_matches_oracle_and_single_grid(cfg):
    b, grids, coeffs, fields, dev, outs = _make_batch(SHAPES)
    lx, ty, st = cfg
    b.set_config(lanes_x=lx, ty=ty, stages=st)
    _run(b, dev, outs)
    info = b.info()
    assert info["cells"] == sum(a * c * d for a, c, d in SHAPES)
    for g, c, f, d, o in zip(grids, coeffs, fields, dev, outs):
        ref = oracle.tendencies(*[x.numpy() for x in f], c)
        got = [g.to_dense(t).numpy() for t in o]
        for x, r in zip(got, ref):
            assert np.abs(interior(x) - interior(r)).max() <= 1e-5 * np.abs(interior(r)).max()
            v = x.copy()
            v[1:-1, 1:-1, 1:-1] = 0
            assert np.all(np.isnan(v[1:-1, 0])) and np.all(np.isnan(v[1:-1, :, 0]))   # halos untouched
        h = pwlib.PW(g, c)
        h.set_tma_config(ty, st, 1, lanes_x=lx)
        single = [g.alloc(fill=NAN) for _ in range(3)]
        h.tendencies(*d, *single)
        h.sync()
        for x, y in zip(o, single):
            assert torch.equal(g.view(x)[1:-1, 1:-1, 1:-1], g.view(y)[1:-1, 1:-1, 1:-1])


def test_batch_graph_replay_and_pointer_change():
    b, grids, coeffs, fields, dev, outs = _make_batch(SHAPES[:4])
    _run(b, dev, outs)
    first = [[t.clone() for t in o] for o in outs]
    for o in outs:
        for t in o:
            t.fill_(NAN)
    _run(b, dev, outs)                     # graph replay, same pointers
    for o, f in zip(outs, first):
        for x, y in zip(o, f):
            assert torch.allclose(x, y, rtol=0, atol=0, equal_nan=True)
    outs2 = [[g.alloc(fill=NAN) for _ in range(3)] for g in grids]
    _run(b, dev, outs2)                    # new pointers: tables re-uploaded
    for o, f in zip(outs2, first):
        for x, y in zip(o, f):
            assert torch.allclose(x, y, rtol=0, atol=0, equal_nan=True)


NARROW = [  # (lanes_x, ty, cells, rows, dtype) -> narrow (lanes_x, cells, ty)
    ((16, 16, 4, 1, "f32"), (8, 4, 32)), ((16, 8, 4, 1, "f32"), (8, 4, 16)), ((32, 8, 4, 1, "f32"), (16, 4, 16)),
    ((8, 16, 8, 3, "bf16"), (8, 4, 16)), ((16, 8, 8, 3, "bf16"), (8, 8, 16)), ((8, 16, 8, 3, "f16"), (8, 4, 16))]
# last columns of every kind: none, narrow only (nx at most half a tile),
# a narrow remainder, a wide remainder, exactly half a tile
NARROW_SHAPES = [(16, 70, 5), (96, 33, 7), (100, 20, 4), (260, 9, 6), (4, 9, 3), (128, 17, 3), (32, 40, 8),
                 (200, 18, 4)]


@pytest.mark.parametrize("case", NARROW, ids=["x".join(map(str, c[0])) for c in NARROW])
def test_batch_narrow_last_columns_same_bits(case):
    """A grid's last column marched with tiles half as wide (the default for
    the shapes that have a narrow partner) gives the bits of the uniform
    tiling and of the single-grid kernel, and the work list holds exactly the
    narrow tiles the tile plan implies."""
    (lx, ty, cells, rows, dtype), (nlx, ncells, nty) = case
    b, grids, coeffs, fields, dev, outs = _make_batch(NARROW_SHAPES, dtype=dtype)
    b.set_config(lanes_x=lx, ty=ty, stages=4, rows=rows, cells=cells)
    assert b.narrow_shape() == {"lanes_x": nlx, "cells": ncells, "ty": nty}
    tw, tn = lx * cells, nlx * ncells
    items = 0
    for nx, ny, _ in NARROW_SHAPES:
        full, r = divmod(nx, tw)
        if 0 < r <= tn:
            items += full * -(-ny // ty) + -(-ny // nty)
        else:
            items += -(-nx // tw) * -(-ny // ty)
    assert b.info()["items"] == items
    _run(b, dev, outs)
    b.set_narrow_columns(False)
    assert b.narrow_shape() == {"lanes_x": 0, "cells": 0, "ty": 0}
    assert b.info()["items"] == sum(-(-nx // tw) * -(-ny // ty) for nx, ny, _ in NARROW_SHAPES)
    outs2 = [[g.alloc(fill=NAN) for _ in range(3)] for g in grids]
    _run(b, dev, outs2)
    def same(g, x, y):   # interiors bit for bit (16-bit: whole arrays, NaN halos included)
        if dtype == "f32":
            return torch.equal(g.view(x)[1:-1, 1:-1, 1:-1], g.view(y)[1:-1, 1:-1, 1:-1])
        return torch.equal(x.view(torch.int16), y.view(torch.int16))

    for g, c, f, d, o, o2 in zip(grids, coeffs, fields, dev, outs, outs2):
        h = pwlib.PW(g, c)
        h.set_tma_config(ty, 4, 1, lanes_x=lx, cells=cells, rows=rows)
        single = [g.alloc(fill=NAN) for _ in range(3)]
        h.tendencies(*d, *single)
        h.sync()
        for x, y, z in zip(o, o2, single):
            assert same(g, x, z) and same(g, x, y)
        if dtype == "f32":
            ref = oracle.tendencies(*[x.numpy() for x in f], c)
            for x, r in zip(o, ref):
                got = g.to_dense(x).numpy()
                assert np.abs(interior(got) - interior(r)).max() <= 1e-5 * np.abs(interior(r)).max()
    b.set_narrow_columns(True)
    assert b.narrow_shape() == {"lanes_x": nlx, "cells": ncells, "ty": nty}


PACKED = [(32, 8, 4, 4, 2), (16, 8, 4, 4, 2), (32, 8, 4, 4, 3), (16, 8, 4, 4, 3), (16, 8, 4, 8, 3),
          (16, 4, 4, 8, 3), (8, 8, 4, 8, 3), (8, 16, 4, 8, 3)]


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("cfg", PACKED, ids=["x".join(map(str, p)) for p in PACKED])
def test_batch_two_rows_per_thread_equals_single_grid(dtype, cfg):
    """16-bit batches in the packed FP32x2 forms (two rows per thread, or one
    row with its cells paired along x) give the bits of the single-grid kernel
    in the same shape, grid by grid (with 8 cells per thread also on grids
    whose nx is 4 mod 8: the last vector of a row stores 4 cells); FP32
    batches reject those shapes."""
    lx, ty, st, cells, rows = cfg
    b, grids, coeffs, fields, dev, outs = _make_batch(SHAPES, dtype=dtype)
    b.set_config(lanes_x=lx, ty=ty, stages=st, rows=rows, cells=cells)
    _run(b, dev, outs)
    for g, c, d, o in zip(grids, coeffs, dev, outs):
        h = pwlib.PW(g, c)
        h.set_tma_config(ty, st, 1, lanes_x=lx, cells=cells, rows=rows)
        single = [g.alloc(fill=NAN) for _ in range(3)]
        h.tendencies(*d, *single)
        h.sync()
        for x, y in zip(o, single):
            assert torch.equal(x.view(torch.int16), y.view(torch.int16))
    b32, *_ = _make_batch(SHAPES[:2])
    with pytest.raises(pwlib.PwError) as e:
        b32.set_config(lanes_x=lx, ty=ty, stages=st, rows=rows, cells=cells)
    assert e.value.status == pwlib.PW_ERR_UNSUPPORTED


@pytest.mark.parametrize("rows", [1, 2])
def test_batch_scaled_fp16_equals_single_grid_and_follows_scale_changes(rows):
    """FP16 batches with power-of-two storage scales give the single-grid
    kernel's bits under the same scales, and a change of scales between calls
    takes effect (the replayed graph is captured again)."""
    shapes = SHAPES[:4]
    b, grids, coeffs, fields, dev, outs = _make_batch(shapes, dtype="f16")
    b.set_config(lanes_x=16, ty=8, stages=4, rows=rows)
    results = []
    for sc in ([1.0] * 6, [0.5, 0.5, 0.5, 8.0, 8.0, 8.0]):
        _run(b, dev, outs, scale=sc)
        results.append([[t.clone() for t in o] for o in outs])
        for g, c, d, o in zip(grids, coeffs, dev, outs):
            h = pwlib.PW(g, c)
            h.set_tma_config(8, 4, 1, lanes_x=16, cells=4, rows=rows)
            single = [g.alloc(fill=NAN) for _ in range(3)]
            h.tendencies(*d, *single, scale=sc)
            h.sync()
            for x, y in zip(o, single):
                assert torch.equal(x.view(torch.int16), y.view(torch.int16))
    # physical in-scale 1/2 and out-scale 8: stored outputs 8 * (1/4) = 2x the unscaled ones
    for a, bb in zip(results[0], results[1]):
        for x, y in zip(a, bb):
            m = torch.isfinite(x) & (x.abs() < 1e4) & (x.abs() > 1e-4)   # no overflow, no subnormals
            assert torch.equal(y[m].float(), 2 * x[m].float())


def test_batch_many_small_grids_bf16():
    shapes = inputs.batch_shapes(n=48, nxy=(32, 160), nzr=(3, 12))
    b, grids, coeffs, fields, dev, outs = _make_batch(shapes, dtype="bf16")
    _run(b, dev, outs)
    for g, c, d, o in zip(grids, coeffs, dev, outs):
        qt = [g.to_dense(t).numpy() for t in d]
        ref = oracle.tendencies(*qt, c)
        a = oracle.abs_terms(*qt, c)
        for x, r, at in zip(o, ref, a):
            got = g.to_dense(x).numpy()
            err = np.abs(interior(got) - interior(r))
            assert np.all(err <= 2.0 ** -8 * np.abs(interior(r)) + 2.0 ** -19 * interior(at) + 1e-30)


def test_batch_rejects_bad_pointers_and_layouts():
    b, grids, coeffs, fields, dev, outs = _make_batch(SHAPES[:2])
    bad = torch.empty(grids[0].alloc_elems + 1, device="cuda")[1:]
    with pytest.raises(pwlib.PwError) as e:
        b.tendencies([bad, dev[1][0]], [d[1] for d in dev], [d[2] for d in dev],
                     [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs])
    assert e.value.status == pwlib.PW_ERR_ALIGN
    g_odd = pwlib.Grid(30, 8, 4)        # nx not a multiple of 4
    with pytest.raises(pwlib.PwError) as e:
        pwlib.Batch([g_odd], [inputs.make_coeffs(4)])
    assert e.value.status == pwlib.PW_ERR_UNSUPPORTED


def test_autotuner_picks_and_caches(tmp_path):
    b, grids, coeffs, fields, dev, outs = _make_batch(SHAPES)
    flds = ([d[0] for d in dev], [d[1] for d in dev], [d[2] for d in dev],
            [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs])
    path = str(tmp_path / "tune.json")
    cfg, times = autotune.tune_batch(b, flds, cache_path=path, reps=2)
    assert len(times) >= 4 and cfg in autotune.BATCH_CANDIDATES
    cfg2, _ = autotune.tune_batch(b, flds, cache_path=path)
    assert cfg2 == cfg
    _run(b, dev, outs)
    for g, c, f, o in zip(grids, coeffs, fields, outs):
        ref = oracle.tendencies(*[x.numpy() for x in f], c)
        for x, r in zip(o, ref):
            got = g.to_dense(x).numpy()
            assert np.abs(interior(got) - interior(r)).max() <= 1e-5 * np.abs(interior(r)).max()
    # single grid
    g, c, d = grids[1], coeffs[1], dev[1]
    h = pwlib.PW(g, c)
    s = [g.alloc() for _ in range(3)]
    gcfg, gt = autotune.tune_grid(h, (*d, *s), cache_path=path, reps=2)
    assert gcfg in autotune.GRID_CANDIDATES and len(gt) >= 4
