"""Parity at the full sizes of the workloads, in the launch configurations the
benchmark times.

* 2048^2 fractal workload: element by element against the FP64 oracle (the
  oracle finishes the full grid in seconds).
* 16384^2 workload: too large for the oracle, so sampled cells.  After N steps
  a cell depends only on the cells within N of it (one face per step), so the
  oracle run on a window of radius N + 2 around a cell, with the GPU's time
  step and closed window edges, gives that cell's exact FP64 value: the edge
  faces reach only N + 1 cells inward in N steps.
* 96-scenario ensemble (256^2 .. 2048^2) on the benchmark's kernel (temporal
  blocking, 4 steps per launch, two launch groups; 128-row base items here,
  the rows per item change no bit): sampled members element by element against
  the oracle run on each alone.

FP32 tolerance: the FP32 path rounds about 6e-8 relative per operation on water
levels of 10-100 m; over these 16-100 steps that stays below 1e-4 m (the
1000-step bound is 1e-3 m).
"""
import dataclasses
import functools

import numpy as np
import pytest

import inputs
from inputs import Options, Problem
import oracle

pytestmark = pytest.mark.gpu

TOL_SHORT = 1e-4
TOL_1000 = 1e-3          # the FP32 bounds after 1000 steps
TOL_MASS = 1e-5


def F():
    import paper_2204_10323_gb300 as F
    return F


def f32(a):
    return None if a is None else a.astype(np.float32).astype(np.float64)


def as_f32(p):
    return Problem(p.name, p.nx, p.ny, p.dx, f32(p.z), f32(p.n), p.sections, p.opts, h0=f32(p.h0), qx0=f32(p.qx0),
                   qy0=f32(p.qy0), steps=p.steps, gauges=p.gauges)


# ---------------------------------------------------------------- 2048^2, element by element
@pytest.mark.parametrize("wet,steps", [(False, 200), (True, 100)])
def test_c2_full_grid_matches_oracle(wet, steps):
    Fm = F()
    p = inputs.c2_fractal()
    if wet:
        p.h0 = inputs.wet_start(p.z, p.dx, 0.3)
    q = as_f32(p)
    o = oracle.Oracle(q)
    o.run(steps)
    s = Fm.Sim(q, precision=Fm.F32)                 # the default kernel (AUTO: temporal blocking) and launch shape
    s.step(steps)
    h, qx, qy = s.state()
    assert np.abs(h.astype(np.float64) - o.h).max() < TOL_SHORT
    assert np.abs(qx.astype(np.float64) - o.qx).max() < 10 * TOL_SHORT
    assert np.abs(qy.astype(np.float64) - o.qy).max() < 10 * TOL_SHORT
    L = s.ledger()
    # the CFL time step of later epochs comes from an FP32 depth maximum
    assert L["t"] == pytest.approx(o.ledger.t, rel=1e-6)
    assert abs(L["volume"] - o.volume()) <= 1e-5 * o.volume()
    s.close()


@pytest.mark.parametrize("wet", [False, True])
def test_c2_full_grid_1000_steps_matches_oracle(wet):
    """The stated bound at the stated length: the full 2048^2 grid, 1000 steps on
    the default kernel, 1e-3 m max-abs depth and 1e-5 relative volume."""
    Fm = F()
    p = inputs.c2_fractal()
    if wet:
        p.h0 = inputs.wet_start(p.z, p.dx, 0.3)
    q = as_f32(p)
    o = oracle.Oracle(q)
    o.run(1000)
    s = Fm.Sim(q, precision=Fm.F32)
    s.step(1000)
    h = s.read(Fm.FIELD_H).astype(np.float64)
    L = s.ledger()
    s.close()
    assert np.abs(h - o.h).max() < TOL_1000
    assert abs(L["volume"] - o.volume()) <= TOL_MASS * o.volume()
    assert L["V_in"] == pytest.approx(o.ledger.V_in, rel=1e-5)
    # water on the grid (the configured dry start fills slowly: the hydrograph peaks at a third of 20000 steps)
    assert (o.h > 0).sum() > (0.25 * o.h.size if wet else 500)


@pytest.mark.parametrize("kernel", [4, 5, 3])
def test_c2_full_grid_vector_friction_matches_oracle(kernel):
    Fm = F()
    p = inputs.c2_fractal()
    p.h0 = inputs.wet_start(p.z, p.dx, 0.3)
    p.opts.friction = 1
    q = as_f32(p)
    o = oracle.Oracle(q)
    o.run(100)
    s = Fm.Sim(q, precision=Fm.F32, kernel=kernel)
    s.step(100)
    h, qx, qy = s.state()
    assert np.abs(h.astype(np.float64) - o.h).max() < TOL_SHORT
    assert np.abs(qx.astype(np.float64) - o.qx).max() < 10 * TOL_SHORT
    assert np.abs(qy.astype(np.float64) - o.qy).max() < 10 * TOL_SHORT
    assert abs(s.ledger()["volume"] - o.volume()) <= 1e-5 * o.volume()
    s.close()


# ---------------------------------------------------------------- 16384^2, sampled cells
@functools.lru_cache(maxsize=1)
def c3_problem():
    return as_f32(inputs.c3_large())


@pytest.fixture(scope="module")
def c3():
    p = c3_problem()
    rng = np.random.default_rng(20405)
    N = 16
    r = N + 2
    wet = np.argwhere(p.h0[r:-r, r:-r] > 0) + r        # cells of the wet region (away from the borders)
    dry = np.argwhere(p.h0[r:-r, r:-r] == 0) + r
    pick = np.concatenate([wet[rng.choice(len(wet), 16, replace=False)],
                           dry[rng.choice(len(dry), 4, replace=False)]])
    return p, N, r, pick


def window_oracle(p, jc, ic, r, dt, steps):
    sl = (slice(jc - r, jc + r + 1), slice(ic - r, ic + r + 1))
    w = Problem("window", 2 * r + 1, 2 * r + 1, p.dx, p.z[sl].copy(), p.n[sl].copy(), [],
                Options(dt_mode=1, dt_const=dt, g=p.opts.g, h_dry=p.opts.h_dry, friction=p.opts.friction),
                h0=p.h0[sl].copy())
    o = oracle.Oracle(w)
    o.run(steps)
    return o


@pytest.mark.parametrize("kernel,k,friction", [(4, 0, 0), (5, 0, 0), (3, 4, 0), (5, 0, 1), (3, 4, 1)])
def test_c3_full_grid_sampled_cells_match_oracle(c3, kernel, k, friction):
    Fm = F()
    p, N, r, pick = c3
    if friction:                                      # the vector-norm friction option (TMA tiles)
        p = dataclasses.replace(p, opts=dataclasses.replace(p.opts, friction=friction))
    s = Fm.Sim(p, precision=Fm.F32, kernel=kernel, steps_per_launch=k)
    s.step(N)                                         # one CFL epoch of 16 steps
    dt = s.ledger()["dt"]
    h = s.read(Fm.FIELD_H)
    qx = s.read(Fm.FIELD_QX)
    s.close()
    moved = 0
    for jc, ic in pick:
        o = window_oracle(p, int(jc), int(ic), r, dt, N)
        assert abs(float(h[jc, ic]) - o.h[r, r]) < TOL_SHORT, (jc, ic)
        assert abs(float(qx[jc, ic]) - o.qx[r, r]) < 10 * TOL_SHORT, (jc, ic)
        moved += abs(o.h[r, r] - p.h0[jc, ic]) > 1e-6
    assert moved >= 4                                 # the samples see water move


def test_c3_full_grid_cells_after_four_epochs_match_oracle():
    """64 steps (four CFL epochs) on the default kernel: windows of radius 66
    around sampled cells, each run by the oracle with the GPU's four epoch time
    steps."""
    Fm = F()
    p = c3_problem()
    N, E = 64, p.opts.epoch_steps
    r = N + 2
    rng = np.random.default_rng(20406)
    wet = np.argwhere(p.h0[r:-r, r:-r] > 0) + r
    dry = np.argwhere(p.h0[r:-r, r:-r] == 0) + r
    pick = np.concatenate([wet[rng.choice(len(wet), 12, replace=False)],
                           dry[rng.choice(len(dry), 4, replace=False)]])
    s = Fm.Sim(p, precision=Fm.F32)
    dts = []
    for _ in range(N // E):
        s.step(E)
        dts.append(s.ledger()["dt"])
    h = s.read(Fm.FIELD_H)
    s.close()
    assert len(set(dts)) > 1                          # the CFL step changes between epochs
    moved = 0
    for jc, ic in pick:
        jc, ic = int(jc), int(ic)
        sl = (slice(jc - r, jc + r + 1), slice(ic - r, ic + r + 1))
        w = Problem("window", 2 * r + 1, 2 * r + 1, p.dx, p.z[sl].copy(), p.n[sl].copy(), [],
                    Options(dt_mode=1, dt_const=dts[0], g=p.opts.g, h_dry=p.opts.h_dry), h0=p.h0[sl].copy())
        o = oracle.Oracle(w)
        for dt in dts:
            for _ in range(E):
                o.step_dt(dt)
        assert abs(float(h[jc, ic]) - o.h[r, r]) < TOL_SHORT, (jc, ic)
        moved += abs(o.h[r, r] - p.h0[jc, ic]) > 1e-6
    assert moved >= 4


# ---------------------------------------------------------------- 96-scenario ensemble
def test_ensemble_96_sampled_members_match_oracle():
    Fm = F()
    probs = []
    for s in range(96):
        p = inputs.c4_scenario(s, steps=5000)
        p.h0 = inputs.wet_start(p.z, p.dx, 0.3)
        probs.append(as_f32(p))
    ens = Fm.Ensemble(probs)
    E = probs[0].opts.epoch_steps
    ens.set_launch(2, 128, 4 * E)
    ens.set_kernel(Fm.KERNEL_TILED, 4)
    steps = 2 * E
    ens.step(steps)
    sizes = [q.nx * q.ny for q in probs]
    order = np.argsort(sizes, kind="stable")
    for m in list(order[:3]) + [int(order[len(order) // 2])]:
        o = oracle.Oracle(probs[m])
        o.run(steps)
        h = ens.members[m].read(Fm.FIELD_H).astype(np.float64)
        assert np.abs(h - o.h).max() < TOL_SHORT, m
    ens.close()


def test_ensemble_96_one_member_of_each_shape_matches_oracle_1024_steps():
    """One member of each of the five grid shapes, 1024 steps (64 epochs) on the
    benchmark's kernel (temporal blocking, K = 4, two launch groups; the rows
    per item change no bit), element by element against the oracle run alone."""
    Fm = F()
    probs = []
    for s in range(96):
        p = inputs.c4_scenario(s, steps=5000)
        p.h0 = inputs.wet_start(p.z, p.dx, 0.3)
        probs.append(as_f32(p))
    ens = Fm.Ensemble(probs)
    E = probs[0].opts.epoch_steps
    ens.set_launch(2, 128, 4 * E)
    ens.set_kernel(Fm.KERNEL_TILED, 4)
    steps = 1024
    ens.step(steps)
    first = {}
    for m, q in enumerate(probs):
        first.setdefault((q.nx, q.ny), m)
    assert len(first) == 5
    for shape, m in sorted(first.items()):
        o = oracle.Oracle(probs[m])
        o.run(steps)
        h = ens.members[m].read(Fm.FIELD_H).astype(np.float64)
        L = ens.members[m].ledger()
        assert np.abs(h - o.h).max() < TOL_1000, (shape, m)
        assert abs(L["volume"] - o.volume()) <= TOL_MASS * o.volume(), (shape, m)
    ens.close()
