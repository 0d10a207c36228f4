"""The synthetic workloads match their stated recipe (CPU).

The paper's DEM, roughness and gauge data are not available, so every
workload is generated from a seed; these tests pin the properties the recipe
promises (grid, spacing, channel, roughness, hydrograph, wet fraction,
sections, determinism) at reduced sizes of the same generators.
"""
import numpy as np
import pytest

import inputs
from inputs import INFLOW, OUTFLOW, XMAX, XMIN, YMIN


def sections_of(p):
    return [(s.side, s.kind) for s in p.sections]


def test_generators_are_deterministic():
    a, b = inputs.c2_fractal(nx=256, ny=256), inputs.c2_fractal(nx=256, ny=256)
    assert np.array_equal(a.z, b.z) and np.array_equal(a.n, b.n)
    c, d = inputs.c4_scenario(7, steps=10), inputs.c4_scenario(7, steps=10)
    assert np.array_equal(c.z, d.z) and np.array_equal(c.n, d.n)
    assert inputs.c4_scenario(8, steps=10).n[0, 0] != c.n[0, 0]     # another scenario, another draw


def test_c1_tilted_channel_recipe():
    p = inputs.c1_tilted_channel()
    assert (p.nx, p.ny, p.dx) == (128, 128, 10.0)
    assert np.all(p.n == 0.03)
    xm = (np.arange(p.nx) + 0.5) * p.dx
    plane = 100.0 - 1e-3 * xm
    drop = plane[None, :] - p.z                       # 3 m in the channel, noise of +-0.1 m elsewhere
    in_chan = drop > 1.5
    assert np.all(in_chan.sum(axis=0) == 8)           # 8 cells wide in every column
    assert np.abs(drop[in_chan] - 3.0).max() <= 0.1 + 1e-12
    assert np.abs(drop[~in_chan]).max() <= 0.1 + 1e-12
    assert sections_of(p) == [(XMIN, INFLOW), (XMAX, OUTFLOW)]
    assert p.sections[0].q_m3s[0] == 50.0 and p.sections[1].frac_start == 0.0 and p.sections[1].frac_end == 1.0
    assert p.h0 is None                               # dry start
    assert p.opts.dt_cap == 2.0 and p.opts.epoch_steps == 16 and p.opts.cfl_alpha == 0.7


def test_c2_fractal_recipe():
    p = inputs.c2_fractal(nx=256, ny=256)
    assert p.dx == 5.0
    assert set(np.unique(p.n)) == {0.035, 0.06}
    chan = p.n == 0.035
    # the carved bed falls monotonically downstream along the channel (running minimum)
    bed = np.where(chan, p.z, np.inf).min(axis=0)
    assert np.all(np.diff(bed) <= 1e-12)
    assert 35.0 < float(p.z.max() - p.z.min()) < 50.0  # 40 m relief plus the 4 m cut
    t, q = p.sections[0].t_s, p.sections[0].q_m3s
    assert q.max() == 800.0 and t[int(np.argmax(q))] == pytest.approx(t[-1] / 3.0)
    assert sections_of(p) == [(XMIN, INFLOW), (XMAX, OUTFLOW)]


def test_c3_large_recipe_at_reduced_size():
    p = inputs.c3_large(nx=512, ny=512)
    assert p.dx == 1.0 and p.opts.dt_cap == 0.1
    assert sections_of(p) == [(XMIN, INFLOW), (YMIN, INFLOW), (XMAX, OUTFLOW)]
    assert all(s.q_m3s.max() == 400.0 for s in p.sections if s.kind == INFLOW)
    wet = float((p.h0 > 0).mean())
    assert 0.25 < wet < 0.35                          # primed to ~30 % wet


def test_c4_ensemble_recipe():
    probs = [inputs.c4_scenario(s, steps=10) for s in range(12)]
    for p in probs:
        assert (p.nx, p.ny) in inputs.ENSEMBLE_SHAPES and p.dx == 5.0
        assert np.all(p.n == p.n[0, 0]) and 0.02 <= p.n[0, 0] <= 0.08
        peak = p.sections[0].q_m3s.max()
        assert 100.0 <= peak <= 1000.0
    assert len({p.n[0, 0] for p in probs}) == len(probs)     # each scenario its own roughness


def test_c5_calibration_recipe():
    p = inputs.c5_calibration(nx=256, ny=256, steps=200)
    assert p.n.min() >= 0.01 and abs(float(p.n.mean()) - 0.04) < 0.01
    truth = inputs.c5_calibration(nx=256, ny=256, steps=200, truth=True)
    assert np.array_equal(truth.z, p.z) and not np.array_equal(truth.n, p.n)   # same terrain, other field
    g = p.gauges
    assert g.shape == (16, 2)
    # gauges sit in the carved channel: below the terrain around them
    z = p.z
    for i, j in g:
        ring = z[max(j - 30, 0):j + 31, i]
        assert z[j, i] <= np.median(ring)
    assert p.opts.dt_mode == 1                        # a fixed dt for the gradient


def test_standing_wave_recipe():
    """Flat closed basin at rest, depth H + eps cos(kx x) cos(ky y) at the cell
    centres: the mode is even about both walls (the cells next to a wall mirror
    the ones at the opposite wall up to the mode's parity) and has zero mean for
    a mode number above 0."""
    p = inputs.standing_wave(12, 10, 2, 3, H=2.0, eps=1e-3, dx=1.5, n=0.03)
    assert (p.nx, p.ny, p.dx) == (12, 10, 1.5) and p.sections == []
    assert not p.z.any() and np.all(p.n == 0.03)
    assert not p.qx0.any() and not p.qy0.any()
    m = (p.h0 - 2.0) / 1e-3
    assert abs(m.max() - 1.0) < 0.1 and abs(m.min() + 1.0) < 0.2
    np.testing.assert_allclose(m[:, ::-1], m, atol=1e-12)          # mx = 2: even under x -> L - x
    np.testing.assert_allclose(m[::-1, :], -m, atol=1e-12)         # my = 3: odd under y -> L - y
    assert abs(m.sum()) < 1e-9
    assert p.opts.dt_mode == 1 and p.opts.dt_const == 0.05
