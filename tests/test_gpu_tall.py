"""Tall grids: launches with more block rows than a CUDA grid's y dimension
holds (65535).  Every 2D-tiled kernel runs a one-dimensional grid and takes
its tile's (x, y) from the block index; these cases pass that limit for the
reference, stream, TMA-tile and adjoint kernels (and run the rows and
temporal-blocking kernels on the same shape), against the FP64 oracle.

Tolerances as in the forward tests: 1e-10 for FP64, 1e-4 m for FP32 over
these 12 steps.
"""
import numpy as np
import pytest

import inputs
from inputs import Problem
import oracle

pytestmark = pytest.mark.gpu

NY = 600_000          # 75000 block rows of 8 (reference, stream/TMA with 8-row chunks)
STEPS = 12


def F():
    import paper_2204_10323_gb300 as F
    return F


def as_f32(p):
    r = lambda a: None if a is None else a.astype(np.float32).astype(np.float64)
    return Problem(p.name, p.nx, p.ny, p.dx, r(p.z), r(p.n), p.sections, p.opts, h0=r(p.h0), qx0=r(p.qx0),
                   qy0=r(p.qy0))


@pytest.fixture(scope="module")
def tall64():
    p = inputs.random_small(3, NY, 31)
    o = oracle.Oracle(p)
    o.run(STEPS)
    return p, o


@pytest.fixture(scope="module")
def tall32():
    p = as_f32(inputs.random_small(3, NY, 31))
    o = oracle.Oracle(p)
    o.run(STEPS)
    return p, o


def test_tall_fp64_reference_matches_oracle(tall64):
    Fm = F()
    p, o = tall64
    s = Fm.Sim(p, precision=Fm.F64)
    s.step(STEPS)
    h, qx, qy = s.state()
    s.close()
    assert np.abs(h - o.h).max() < 1e-10
    assert np.abs(qx - o.qx).max() < 1e-10
    assert np.abs(qy - o.qy).max() < 1e-10
    assert np.abs(o.h - p.h0).max() > 1e-4          # water moved


@pytest.mark.parametrize("kernel,k,tile", [(4, 0, (1, 8)), (5, 0, (1, 8)), (1, 0, (0, 0)), (2, 0, (0, 0)),
                                           (3, 4, (0, 0))])
def test_tall_fp32_kernels_match_oracle(tall32, kernel, k, tile):
    Fm = F()
    p, o = tall32
    s = Fm.Sim(p, precision=Fm.F32, kernel=kernel, steps_per_launch=k, tile=tile)
    s.step(STEPS)
    h, qx, qy = s.state()
    L = s.ledger()
    s.close()
    assert np.abs(h.astype(np.float64) - o.h).max() < 1e-4
    assert np.abs(qx.astype(np.float64) - o.qx).max() < 1e-3
    assert np.abs(qy.astype(np.float64) - o.qy).max() < 1e-3
    assert abs(L["volume"] - o.volume()) <= 1e-5 * o.volume()


def test_tall_fp64_adjoint_matches_oracle():
    Fm = F()
    p = inputs.random_small(2, NY, 32)
    steps = 5
    gauges = np.array([[0, 10], [1, NY // 2], [0, NY - 3]])
    w = np.random.default_rng(9).standard_normal((steps, len(gauges)))
    gn_o = oracle.Oracle(p).adjoint(steps, gauges, w)
    s = Fm.Sim(p, precision=Fm.F64)
    gn = s.adjoint(steps, gauges, w, n_checkpoints=steps)
    s.close()
    scale = np.abs(gn_o).max()
    assert scale > 0
    assert np.abs(gn - gn_o).max() <= 1e-9 * scale
