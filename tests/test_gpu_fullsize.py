"""Parity at the benchmark's full sizes, in the launch shapes the benchmark
times, where the plain FP32 full-size check (test_gpu_tendencies) does not
reach:

  * 16-bit storage at 2048 x 2048 x 64 (automatic shape: 8 cells per
    thread packed as FP32x2 pairs along x) on sampled 32 x 32-column boxes,
    against the per-cell kernel and total bounds of the 16-bit tests;
  * the 512-grid batch (1.77 G cells) in the autotuner's tile, 8 sampled grids
    (largest and smallest among them) checked whole against the FP64 oracle;
  * the periodic adjoint at 512 x 512 x 64 (the rollout's grid) through the
    identity <J(q) d, l> = <d, J(q)^T l>, with J(q) d = s(q + d) - s(q) - s(d)
    (s is quadratic) evaluated by the forward kernel and both sums in FP64.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2301_13016_gb300 as pwlib
from paper_2301_13016_gb300 import inputs, precision
from gpu_util import NAN, interior

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _boxes(nx, ny, n, seed=1):
    rng = np.random.default_rng(seed)
    b = [(1, 1), (1, nx - n + 1), (ny - n + 1, 1), (ny - n + 1, nx - n + 1)]
    return b + [(int(rng.integers(1, ny - n)), int(rng.integers(1, nx - n))) for _ in range(4)]


def _sub(f, j0, i0, n):
    """dense sub-array with one halo cell around rows j0.., columns i0.. (all levels)"""
    return f[:, j0 - 1:j0 + n + 1, i0 - 1:i0 + n + 1]


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_16bit_sampled_parity_2048(dtype):
    nx = ny = 2048
    nz = 64
    c = inputs.make_coeffs(nz)
    f = inputs.random_fields(nx, ny, nz, device="cuda")
    sc = precision.suggest_scales([float(x.abs().max()) for x in f], c, dtype)
    g = pwlib.Grid(nx, ny, nz, dtype=dtype)
    h = pwlib.PW(g, c)
    assert h.tma_config()["rows"] == 3 and h.tma_config()["cells"] == 8   # the benchmark's 16-bit shape
    dev = [g.from_dense(x, scale=s) for x, s in zip(f, sc[:3])]
    outs = [g.alloc(fill=NAN) for _ in range(3)]
    h.tendencies(*dev, *outs, scale=sc)
    h.sync()
    assert h.last_kernel == 2
    us = precision.UNIT_ROUNDOFF[dtype]
    n = 32
    qv = [g.view(d) for d in dev]
    ov = [g.view(o) for o in outs]
    for j0, i0 in _boxes(nx, ny, n):
        qt = [_sub(v, j0, i0, n).double().cpu().numpy() * s for v, s in zip(qv, sc[:3])]   # dequantised inputs
        q = [_sub(x, j0, i0, n).double().cpu().numpy() for x in f]                          # the FP32 fields
        got = [_sub(v, j0, i0, n)[1:-1, 1:-1, 1:-1].double().cpu().numpy() / s for v, s in zip(ov, sc[3:])]
        ref_t, a_t = oracle.tendencies(*qt, c), oracle.abs_terms(*qt, c)
        ref, a_q = oracle.tendencies(*q, c), oracle.abs_terms(*q, c)
        for x, rt, at, r, aq, so in zip(got, ref_t, a_t, ref, a_q, sc[3:]):
            floor = 2 * precision.MIN_NORMAL[dtype] / so
            assert np.all(np.abs(x - interior(rt)) <= us * np.abs(interior(rt)) + 2.0 ** -19 * interior(at) + floor)
            assert np.all(np.abs(x - interior(r)) <=
                          us * np.abs(interior(r)) + (2 * us + 2.0 ** -19) * interior(aq) * 1.05 + floor)


def test_batch_512_grids_sampled():
    shapes = inputs.batch_shapes()
    grids, coeffs, dev, outs = [], [], [], []
    for q, (nx, ny, nz) in enumerate(shapes):
        g = pwlib.Grid(nx, ny, nz)
        grids.append(g)
        coeffs.append(inputs.make_coeffs(nz))
        d = inputs.random_fields(nx, ny, nz, device="cuda", seeds=(10 + 3 * q, 11 + 3 * q, 12 + 3 * q))
        dev.append([g.from_dense(x) for x in d])
        outs.append([g.alloc(fill=NAN) for _ in range(3)])
        del d
    b = pwlib.Batch(grids, coeffs)
    b.set_config(lanes_x=16, ty=4, stages=4)
    b.tendencies([x[0] for x in dev], [x[1] for x in dev], [x[2] for x in dev],
                 [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs])
    b.sync()
    cells = [nx * ny * nz for nx, ny, nz in shapes]
    rng = np.random.default_rng(7)
    pick = {int(np.argmax(cells)), int(np.argmin(cells))} | set(int(x) for x in rng.choice(len(shapes), 6, replace=False))
    for q in sorted(pick):
        g = grids[q]
        ins = [g.to_dense(t).numpy() for t in dev[q]]
        ref = oracle.tendencies(*ins, coeffs[q])
        for o, r in zip(outs[q], ref):
            got = g.to_dense(o).numpy()
            assert np.abs(interior(got) - interior(r)).max() <= TOL * np.abs(interior(r)).max(), (q, shapes[q])
    del dev, outs, b
    torch.cuda.empty_cache()


def test_adjoint_dot_product_512():
    nx = ny = 512
    nz = 64
    c = inputs.make_coeffs(nz)
    g = pwlib.Grid(nx, ny, nz)
    h = pwlib.PW(g, c)
    q = [g.from_dense(x) for x in inputs.smooth_fields(nx, ny, nz, w_zero=True, device="cuda")]
    d = [g.from_dense(x) for x in inputs.random_fields(nx, ny, nz, device="cuda", seeds=(31, 32, 33))]
    lam = [g.from_dense(x) for x in inputs.random_fields(nx, ny, nz, device="cuda", seeds=(34, 35, 36))]
    qd = [a + b for a, b in zip(q, d)]
    for t in q + d + qd:
        h.fill_halo_periodic(t)

    def tend(fields):
        out = [g.alloc(fill=0.0) for _ in range(3)]
        h.tendencies(*fields, *out)
        return out

    s_qd, s_q, s_d = tend(qd), tend(q), tend(d)
    gr = [g.alloc(fill=NAN) for _ in range(3)]
    h.adjoint(*q, *lam, *gr, alpha=1.0, flags=pwlib.PW_ADJ_PERIODIC)
    h.sync()
    assert h.last_kernel == 2
    inner = lambda t: g.view(t)[1:-1, 1:-1, 1:-1].double()
    # the scheme's outputs: su, sv at levels 2..nz, sw at 2..nz-1 (level index k is k-1 in `inner`)
    lv = [slice(1, nz), slice(1, nz), slice(1, nz - 1)]
    lhs = sum(float(((inner(a) - inner(b) - inner(e))[k] * inner(l)[k]).sum())
              for a, b, e, l, k in zip(s_qd, s_q, s_d, lam, lv))
    rhs = sum(float((inner(x) * inner(y)).sum()) for x, y in zip(d, gr))
    assert abs(lhs - rhs) <= 1e-4 * abs(rhs), (lhs, rhs)
