"""Failure detection on the host side, without a GPU fault.

* Allocation failure: the library's allocation hook makes its k-th device
  allocation fail; for every k of flood_create, of flood_adjoint's snapshot
  store, of flood_ensemble_create and of flood_decomp_create the call returns
  FLOOD_ERR_OOM and PyTorch's allocator holds exactly what it held before.
* Pitch padding: the padding of every grid plane is filled with NaNs of a
  fixed bit pattern; after steps on each kernel family no padding element has
  changed (no kernel writes there) and the state equals an unpoisoned run bit
  for bit (no result reads there).
"""
import dataclasses

import numpy as np
import pytest

import inputs
from inputs import Problem

pytestmark = pytest.mark.gpu


def F():
    import paper_2204_10323_gb300 as F
    return F


def allocated():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.memory_allocated()


def f32(p):
    r = lambda a: None if a is None else a.astype(np.float32).astype(np.float64)
    return Problem(p.name, p.nx, p.ny, p.dx, r(p.z), r(p.n), p.sections, p.opts, h0=r(p.h0), qx0=r(p.qx0),
                   qy0=r(p.qy0))


def sweep_failures(make, check_after=None):
    """make() once to count its allocations, then make it fail at each of them."""
    Fm = F()
    base = allocated()
    n0 = Fm.flood_debug_alloc_count()
    obj = make()
    n_alloc = Fm.flood_debug_alloc_count() - n0
    obj.close()
    assert allocated() == base
    assert n_alloc >= 3
    try:
        for k in range(n_alloc):
            Fm.flood_debug_fail_alloc_after(k)
            with pytest.raises(Fm.FloodError) as e:
                make()
            assert e.value.status == Fm.ERR_OOM, (k, e.value)
            assert allocated() == base, k
            if check_after:
                check_after()
    finally:
        Fm.flood_debug_fail_alloc_after(-1)
    return n_alloc


@pytest.mark.parametrize("precision", [0, 1])
def test_create_fails_cleanly_at_every_allocation(precision):
    Fm = F()
    p = inputs.random_small(40, 23, 5)
    n = sweep_failures(lambda: Fm.Sim(p, precision=precision))
    assert n >= 20
    s = Fm.Sim(p, precision=precision)             # the library works afterwards
    s.step(8)
    s.sync()
    s.close()


def test_adjoint_snapshot_store_fails_cleanly():
    Fm = F()
    p = f32(inputs.random_small(40, 23, 5))
    s = Fm.Sim(p)
    g = np.array([[5, 5], [20, 12]])
    seed = np.ones((24, 2))
    ref = s.adjoint(24, g, seed, n_checkpoints=4)
    h0 = s.read(Fm.FIELD_H)

    class Call:                                     # one adjoint sweep, shaped like a created object
        def __init__(self):
            self.gn = s.adjoint(24, g, seed, n_checkpoints=4)

        def close(self):
            pass

    n = sweep_failures(Call)
    assert n >= 10                                  # snapshots, logs, adjoint planes
    assert np.array_equal(Call().gn, ref)           # the handle is intact: same gradient, same state
    assert np.array_equal(s.read(Fm.FIELD_H), h0)
    s.close()


def test_ensemble_create_fails_cleanly():
    Fm = F()
    probs = [f32(inputs.random_small(40, 23, 5)), f32(inputs.random_small(33, 17, 1)),
             f32(inputs.random_small(70, 41, 2))]
    n = sweep_failures(lambda: Fm.Ensemble(probs))
    assert n >= 3 * 20


def test_decomp_create_fails_cleanly():
    Fm = F()
    p = inputs.random_small(40, 23, 5)
    n = sweep_failures(lambda: Fm.Decomp(p, 3, 2, precision=Fm.F64))
    assert n >= 3 * 20


def test_hook_turns_itself_off():
    Fm = F()
    p = inputs.random_small(20, 12, 2)
    Fm.flood_debug_fail_alloc_after(0)
    with pytest.raises(Fm.FloodError):
        Fm.Sim(p)
    Fm.Sim(p).close()                               # the next create succeeds
    Fm.flood_debug_fail_alloc_after(5)
    Fm.flood_debug_fail_alloc_after(-1)             # and an armed hook can be turned off
    Fm.Sim(p).close()


# ---------------------------------------------------------------- pitch padding
@pytest.mark.parametrize("shape", [(37, 29), (130, 70)])
@pytest.mark.parametrize("precision,kernel,k,theta,friction", [
    (1, 1, 0, 1.0, 0), (0, 1, 0, 1.0, 0), (0, 2, 0, 1.0, 0), (0, 4, 0, 1.0, 0), (0, 5, 0, 1.0, 0),
    (0, 3, 4, 1.0, 0), (0, 3, 8, 1.0, 0), (0, 4, 0, 0.9, 1), (0, 5, 0, 0.9, 1), (1, 1, 0, 0.9, 1)])
def test_padding_is_never_written_and_never_read(shape, precision, kernel, k, theta, friction):
    Fm = F()
    p = inputs.random_small(shape[0], shape[1], 3)
    p.opts = dataclasses.replace(p.opts, theta=theta, friction=friction, epoch_steps=8)
    q = p if precision == 1 else f32(p)
    ref = Fm.Sim(q, precision=precision, kernel=kernel, steps_per_launch=k)
    ref.step(64)
    ref.sync()
    want = ref.state()
    ref.close()
    s = Fm.Sim(q, precision=precision, kernel=kernel, steps_per_launch=k)
    Fm.flood_debug_padding(s.h, True)
    assert Fm.flood_debug_padding(s.h, False) == 0
    s.step(64)
    s.sync()
    assert Fm.flood_debug_padding(s.h, False) == 0
    got = s.state()
    for a, b in zip(want, got):
        assert np.array_equal(a, b)
    s.close()
