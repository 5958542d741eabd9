"""Parity at the two workloads that run many steps, at their stated sizes.

  * 100 fused forward-Euler steps (dt = 1 s) on 2048 x 2048 x 64 with FP32,
    BF16 and FP16 state, one and two steps per pass, on the smooth field with
    w = 0 initially (the literal random field diverges: forward Euler with an
    energy-conserving scheme grows ||q||^2 by dt^2 ||s||^2 every step).  The
    error against the FP64 oracle is taken every 10 steps on sampled 32 x 32
    columns (all levels).  The scheme reaches one cell further per step, so
    the oracle runs on the box of 32 + 2 * 101 columns around each sample
    (taken with the periodic wrap from the GPU's own start state): whatever
    enters the box through its edges reaches at most 100 cells in by step
    100, so the centre 32 x 32 is exact.
  * The differentiable 20-step rollout on 512 x 512 x 64 FP32 with a
    checkpoint every 5 steps and the loss 0.5 * sum((u_T - u_target)^2): the
    whole gradient against the oracle's FP64 reverse sweep, and the
    derivative along a direction supported on an 8^3 sub-box against central
    differences with eps = 1e-3.

Run as a script (python tests/test_gpu_configs.py) on a GPU it prints the
per-10-step error table of the 100-step run.
"""
import concurrent.futures as cf
import math
import os
import sys

import numpy as np
import pytest
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
if os.path.dirname(HERE) not in sys.path:
    sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
import paper_2301_13016_gb300 as pwlib  # noqa: E402
from paper_2301_13016_gb300 import inputs, precision  # noqa: E402
from paper_2301_13016_gb300.autograd import rollout  # noqa: E402

pytestmark = pytest.mark.gpu

NX = NY = 2048
NZ = 64
NSTEPS, EVERY, DT = 100, 10, 1.0
NBOX = 32                 # sampled columns per side
MARGIN = NSTEPS + 1       # cells of the oracle box beyond the sample on each side
SAMPLES = [(1, 1), (1000, 1337), (NY - NBOX + 1, NX - NBOX - 40)]   # (j0, i0): a corner (wraps), inside, an edge
F32_BAR = 1e-5


def _wrapped(start, count, n):
    """1-based indices start .. start+count-1 wrapped onto 1..n."""
    return (np.arange(start, start + count) - 1) % n + 1


def _gather(grid, t, j0, i0, nj, ni, scale):
    """Levels 0..nz+1, rows j0..j0+nj-1 and columns i0..i0+ni-1 (1-based,
    wrapped periodically) of a device field, as float64 physical values."""
    v = grid.view(t)
    h = grid.halo
    jj = torch.as_tensor(_wrapped(j0, nj, grid.ny) + h - 1, device=t.device)
    ii = torch.as_tensor(_wrapped(i0, ni, grid.nx) + h - 1, device=t.device)
    return (v.index_select(1, jj).index_select(2, ii).double() * scale).cpu().numpy()


def _oracle_boxes(start_boxes, c):
    """FP64 rollouts of each sample's box: per sample the centre NBOX x NBOX
    columns of (u, v, w) after every EVERY steps."""
    def run(box):
        q = [np.ascontiguousarray(x) for x in box]
        out = []
        for _ in range(NSTEPS // EVERY):
            q = list(oracle.step(*q, c, DT, EVERY))
            s = slice(1 + MARGIN, 1 + MARGIN + NBOX)
            out.append([x[1:-1, s, s].copy() for x in q])
        return out
    with cf.ThreadPoolExecutor(max_workers=len(start_boxes)) as ex:   # the C oracle runs outside the GIL
        return list(ex.map(run, start_boxes))


def _rel(got, ref, uref):
    """max|err| / max|ref| for u and v; w (zero at the start, grown from the
    u, v coupling) against the u scale."""
    e = [float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)) for a, b in zip(got[:2], ref[:2])]
    e.append(float(np.abs(got[2] - ref[2]).max() / np.abs(uref).max()))
    return max(e)


def rollout_errors(dtype, spp, c=None, fields=None):
    """The 100-step run of one state dtype with spp steps per pass: the
    largest relative error over the sampled columns after every EVERY steps
    (a list of NSTEPS // EVERY values)."""
    c = c if c is not None else inputs.make_coeffs(NZ)
    f = fields if fields is not None else inputs.smooth_fields(NX, NY, NZ, w_zero=True, device="cuda")
    sc = [1.0, 1.0, 1.0]
    if dtype != "f32":
        sc = precision.suggest_scales([max(float(x.abs().max()), 1.0) for x in f], c, dtype)[:3]
    g = pwlib.Grid(NX, NY, NZ, dtype=dtype, halo=spp)
    h = pwlib.PW(g, c)
    h.set_step_blocking(spp)
    q = [g.from_dense(x, scale=s) for x, s in zip(f, sc)]
    tmp = [g.alloc() for _ in range(3)]
    for t in q:
        h.fill_halo_periodic(t)
    h.sync()
    nb = NBOX + 2 * MARGIN
    # the oracle starts from the GPU's own (stored, then scaled) start state
    starts = [[_gather(g, t, j0 - MARGIN - 1, i0 - MARGIN - 1, nb + 2, nb + 2, s) for t, s in zip(q, sc)]
              for j0, i0 in SAMPLES]
    refs = _oracle_boxes(starts, c)
    errs = []
    for n in range(NSTEPS // EVERY):
        h.step(*q, *tmp, DT, EVERY, scale=sc if dtype != "f32" else None)
        h.sync()
        assert h.last_kernel == (3 if spp == 2 else 2)
        e = 0.0
        for (j0, i0), ref in zip(SAMPLES, refs):
            got = [_gather(g, t, j0, i0, NBOX, NBOX, s)[1:-1] for t, s in zip(q, sc)]
            e = max(e, _rel(got, ref[n], ref[n][0]))
        errs.append(e)
    del q, tmp
    torch.cuda.empty_cache()
    return errs


def bar(dtype, spp, steps):
    """FP32: the 1e-5 bar.  16-bit state: the state is rounded to the
    storage format once per pass, an error of at most one unit roundoff u_s
    of the state each time; the stated bound allows 1.5 u_s per rounding (the
    dynamics carries earlier errors along) over the passes taken."""
    if dtype == "f32":
        return F32_BAR
    return 1.5 * precision.UNIT_ROUNDOFF[dtype] * math.ceil(steps / spp)


@pytest.fixture(scope="module")
def smooth_2048():
    c = inputs.make_coeffs(NZ)
    return c, inputs.smooth_fields(NX, NY, NZ, w_zero=True, device="cuda")


@pytest.mark.parametrize("spp", [1, 2], ids=["one_step_per_pass", "two_steps_per_pass"])
@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_100_steps_2048_sampled(smooth_2048, dtype, spp):
    c, f = smooth_2048
    errs = rollout_errors(dtype, spp, c, f)
    for n, e in enumerate(errs):
        assert e <= bar(dtype, spp, (n + 1) * EVERY), (n, errs)


# ---------------------------------------------------------------------------
# The 20-step rollout gradient on 512 x 512 x 64 (checkpoint every 5 steps).

RX = RY = 512
RZ = 64
RSTEPS, REVERY = 20, 5


def _loss_terms(g, uT, ut):
    """Per-cell terms 0.5 * (u_T - u_target)^2 in FP64 (interior cells)."""
    d = g.view(uT)[1:-1, 1:-1, 1:-1].double() - ut[1:-1, 1:-1, 1:-1].to(uT.device).double()
    return 0.5 * d * d


@pytest.fixture(scope="module")
def rollout_512():
    c = inputs.make_coeffs(RZ)
    f = inputs.smooth_fields(RX, RY, RZ, w_zero=True)
    g = pwlib.Grid(RX, RY, RZ)
    h = pwlib.PW(g, c)
    q0 = [g.from_dense(x).requires_grad_(True) for x in f]
    ut = inputs.target_field(RX, RY, RZ)
    uT, vT, wT = rollout(*q0, h, DT, RSTEPS, REVERY)
    L = _loss_terms(g, uT, ut).sum()
    L.backward()
    return c, f, g, h, q0, ut


def test_rollout_gradient_512_matches_oracle(rollout_512):
    """The whole gradient of the 20-step rollout against the oracle's FP64
    forward run and reverse sweep from the same FP32 start (1e-4 of the
    largest gradient entry: the GPU runs the forward steps in FP32)."""
    c, f, g, h, q0, ut = rollout_512
    qT = oracle.step(*[x.numpy() for x in f], c, DT, RSTEPS)
    gT = np.zeros(qT[0].shape)
    gT[1:-1, 1:-1, 1:-1] = qT[0][1:-1, 1:-1, 1:-1] - ut.numpy()[1:-1, 1:-1, 1:-1]
    del qT
    ref = oracle.step_adjoint(*[x.numpy() for x in f], c, DT, RSTEPS, gT, np.zeros_like(gT), np.zeros_like(gT))
    for t, r in zip(q0, ref):
        got = g.to_dense(t.grad).numpy()
        assert np.abs(got[1:-1, 1:-1, 1:-1] - r[1:-1, 1:-1, 1:-1]).max() <= 1e-4 * np.abs(r).max()
        assert np.all(got[:, 0] == 0) and np.all(got[:, :, 0] == 0)     # halo entries carry no gradient


def test_rollout_gradient_512_central_differences(rollout_512):
    """dL/de along a direction d supported on an 8^3 sub-box: central
    differences with eps = 1e-3 of the GPU rollout against <grad, d>.  The
    loss difference L(q + eps d) - L(q - eps d) is summed cell by cell in
    FP64, so the cells the perturbation never reaches (bit-identical in the
    two runs) add exactly zero."""
    c, f, g, h, q0, ut = rollout_512
    gen = torch.Generator().manual_seed(4)
    d = []
    for n in range(3):
        x = torch.zeros((RZ + 2, RY + 2, RX + 2))
        x[20:28, 200:208, 300:308] = torch.randn((8, 8, 8), generator=gen)
        d.append(x)
    dd = [g.from_dense(x) for x in d]
    ana = sum(float((t.grad.double() * e.double()).sum()) for t, e in zip(q0, dd))
    eps = 1e-3

    def terms_at(s):
        with torch.no_grad():
            q = [(t.detach() + s * e) for t, e in zip(q0, dd)]
            out = rollout(*q, h, DT, RSTEPS, REVERY)
            return _loss_terms(g, out[0], ut)

    fd = float((terms_at(eps) - terms_at(-eps)).sum()) / (2 * eps)
    assert abs(fd - ana) <= 1e-3 * abs(ana), (fd, ana)


if __name__ == "__main__":
    c = inputs.make_coeffs(NZ)
    f = inputs.smooth_fields(NX, NY, NZ, w_zero=True, device="cuda")
    rows = {}
    for dtype, spp in (("f32", 1), ("f32", 2), ("bf16", 1), ("bf16", 2), ("f16", 1), ("f16", 2)):
        rows[(dtype, spp)] = rollout_errors(dtype, spp, c, f)
    print("| state | " + " | ".join(str((n + 1) * EVERY) for n in range(NSTEPS // EVERY)) + " |")
    print("|---|" + "---|" * (NSTEPS // EVERY))
    for (dtype, spp), e in rows.items():
        name = f"{dtype} state, {'one step' if spp == 1 else 'two steps'} per pass"
        print(f"| {name} | " + " | ".join(f"{x:.2e}" for x in e) + " |")
    print("bound after 100 steps: " + ", ".join(f"{d}/{s}: {bar(d, s, NSTEPS):.3g}" for d, s in rows))
