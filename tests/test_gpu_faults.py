"""Failure handling with failures injected on the host (pw_inject_failures):
an allocation or a TMA descriptor encoding that fails makes the entry point
return its error, leaves the handle or batch as it was, and the next call
succeeds with correct results.  Nothing reaches the GPU: the injected
failures happen before any CUDA call, so no kernel ever sees a missing
buffer or descriptor."""
import numpy as np
import pytest
import torch

import oracle
import paper_2301_13016_gb300 as pwlib
from paper_2301_13016_gb300 import inputs
from gpu_util import NAN, interior, setup

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _clear_injection():
    yield
    pwlib.inject_failures(pwlib.INJECT_ALLOC, 0)
    pwlib.inject_failures(pwlib.INJECT_TENSOR_MAP, 0)


def _close(got, ref, tol=1e-5):
    return np.abs(interior(got) - interior(ref)).max() <= tol * np.abs(interior(ref)).max()


def test_create_fails_cleanly_then_succeeds():
    g = pwlib.Grid(64, 16, 8)
    c = inputs.make_coeffs(8)
    pwlib.inject_failures(pwlib.INJECT_ALLOC, 1)
    with pytest.raises(pwlib.PwError) as e:
        pwlib.PW(g, c)
    assert e.value.status == pwlib.PW_ERR_OOM
    h = pwlib.PW(g, c)                      # the one injected failure was consumed
    f = inputs.random_fields(64, 16, 8)
    d = [g.from_dense(x) for x in f]
    o = [g.alloc(fill=NAN) for _ in range(3)]
    h.tendencies(*d, *o)
    h.sync()
    for x, r in zip(o, oracle.tendencies(*[t.numpy() for t in f], c)):
        assert _close(g.to_dense(x).numpy(), r)


def test_host_path_staging_allocation_failure():
    c, f, g, h, dev, outs = setup(96, 20, 10)
    hin = [torch.zeros(g.alloc_elems, dtype=torch.float32) for _ in range(3)]
    for a, t in zip(hin, dev):
        a.copy_(t.cpu())
    hout = [torch.full((g.alloc_elems,), NAN, dtype=torch.float32) for _ in range(3)]
    pwlib.inject_failures(pwlib.INJECT_ALLOC, 1)
    with pytest.raises(pwlib.PwError) as e:
        h.tendencies_host(*hin, *hout)
    assert e.value.status == pwlib.PW_ERR_OOM
    h.tendencies_host(*hin, *hout)          # staging allocated now
    ref = oracle.tendencies(*[x.numpy() for x in f], c)
    for x, r in zip(hout, ref):
        assert _close(g.to_dense(x).numpy(), r)


def test_scratch_allocation_failure_of_the_weighted_dot():
    c, f, g, h, dev, outs = setup(64, 12, 6)
    pwlib.inject_failures(pwlib.INJECT_ALLOC, 1)
    with pytest.raises(pwlib.PwError) as e:
        h.weighted_dot(dev[0], dev[1])
    assert e.value.status == pwlib.PW_ERR_OOM
    a = h.weighted_dot(dev[0], dev[1])
    b = h.weighted_dot(dev[0], dev[1])
    assert a == b and np.isfinite(a)


def test_tensor_map_failure_then_success():
    c, f, g, h, dev, outs = setup(256, 24, 12)
    pwlib.inject_failures(pwlib.INJECT_TENSOR_MAP, 1)
    with pytest.raises(pwlib.PwError) as e:
        h.tendencies(*dev, *outs)
    assert e.value.status == pwlib.PW_ERR_CUDA
    h.sync()
    for o in outs:                          # nothing was launched
        assert torch.isnan(g.view(o)[1:-1, 1:-1, 1:-1]).all()
    h.tendencies(*dev, *outs)
    h.sync()
    assert h.last_kernel == 2
    for x, r in zip(outs, oracle.tendencies(*[t.numpy() for t in f], c)):
        assert _close(g.to_dense(x).numpy(), r)


def _batch(shapes):
    grids, coeffs, fields, dev = [], [], [], []
    for q, (nx, ny, nz) in enumerate(shapes):
        g = pwlib.Grid(nx, ny, nz)
        c = inputs.make_coeffs(nz)
        f = inputs.random_fields(nx, ny, nz, seeds=(40 + 3 * q, 41 + 3 * q, 42 + 3 * q))
        grids.append(g)
        coeffs.append(c)
        fields.append(f)
        dev.append([g.from_dense(x) for x in f])
    return grids, coeffs, fields, dev


def _run(b, dev, outs):
    b.tendencies([d[0] for d in dev], [d[1] for d in dev], [d[2] for d in dev],
                 [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs])
    b.sync()


def test_batch_failures_leave_the_batch_usable():
    """A batch whose creation fails is not returned; a work-list rebuild that
    fails keeps the previous shape, work list and graph; a descriptor
    encoding that fails keeps the tables; each next call succeeds."""
    shapes = [(96, 20, 6), (260, 9, 5), (32, 40, 4)]
    grids, coeffs, fields, dev = _batch(shapes)
    pwlib.inject_failures(pwlib.INJECT_ALLOC, 1)
    with pytest.raises(pwlib.PwError) as e:
        pwlib.Batch(grids, coeffs)
    assert e.value.status == pwlib.PW_ERR_OOM
    b = pwlib.Batch(grids, coeffs)
    b.set_config(lanes_x=16, ty=16, stages=4)
    outs = [[g.alloc(fill=NAN) for _ in range(3)] for g in grids]
    _run(b, dev, outs)                      # graph captured for 16 x 16 tiles
    before = b.info()
    pwlib.inject_failures(pwlib.INJECT_ALLOC, 1)
    with pytest.raises(pwlib.PwError) as e:
        b.set_config(lanes_x=32, ty=4, stages=4)
    assert e.value.status == pwlib.PW_ERR_OOM
    assert b.info() == before               # still the 16 x 16 work list
    assert b.narrow_shape() == {"lanes_x": 8, "cells": 4, "ty": 32}
    pwlib.inject_failures(pwlib.INJECT_ALLOC, 1)
    with pytest.raises(pwlib.PwError):
        b.set_narrow_columns(False)
    assert b.narrow_shape() == {"lanes_x": 8, "cells": 4, "ty": 32}
    outs2 = [[g.alloc(fill=NAN) for _ in range(3)] for g in grids]
    pwlib.inject_failures(pwlib.INJECT_TENSOR_MAP, 1)
    with pytest.raises(pwlib.PwError) as e:
        _run(b, dev, outs2)                 # new pointers: the tables are rebuilt, and that fails
    assert e.value.status == pwlib.PW_ERR_CUDA
    for o in outs2:
        for t in o:
            assert torch.isnan(t).all()     # nothing was launched
    _run(b, dev, outs2)
    for g, c, f, o, o1 in zip(grids, coeffs, fields, outs2, outs):
        ref = oracle.tendencies(*[x.numpy() for x in f], c)
        for x, x1, r in zip(o, o1, ref):
            assert _close(g.to_dense(x).numpy(), r)
            assert torch.equal(g.view(x)[1:-1, 1:-1, 1:-1], g.view(x1)[1:-1, 1:-1, 1:-1])
