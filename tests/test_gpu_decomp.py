"""Domain decomposition (1 x N row strips with halo exchange; Methods, "TPU
Implementation") against the single grid, through the C ABI.

A part's kernels see walls at its cut ends, and a wall spoils one more row of
the part per step (the stencil of Eq. 3-4 reaches one cell), so after `halo`
steps the part's own rows are still computed from exactly the inputs the
whole grid uses, by the same kernel arithmetic: the assembled state must be
bitwise the single grid's, and so must the time, the time step and the step
count (the epoch's h_max is an exact maximum).  The inflow volume is booked by
part 0 alone from the same Eq. 6 discharges, so it is bitwise too.  The
outflow and clipped volumes and the stored volume are sums whose order
changes with the split: FP64 within 1e-12 of the ledger's scale, FP32 (whose
temporal-blocking kernel folds float partial sums over runs of rows) within
1e-6; the stored volume (two-sum per thread, double across threads) within
1e-10 either way.
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


def f32(a):
    return None if a is None else a.astype(np.float32).astype(np.float64)


def as_f32(p):
    return Problem(p.name, p.nx, p.ny, p.dx, f32(p.z), f32(p.n), p.sections, p.opts, h0=f32(p.h0), qx0=f32(p.qx0),
                   qy0=f32(p.qy0), steps=p.steps, gauges=p.gauges)


def run(sim, steps):
    sim.step(steps)
    sim.sync()
    out = sim.state(), sim.ledger()
    sim.close()
    return out


def compare(single, dec, rel_sum, rel_vol=1e-10):
    (h1, qx1, qy1), L1 = single
    (h2, qx2, qy2), L2 = dec
    assert np.array_equal(h1, h2), float(np.abs(h1.astype(np.float64) - h2).max())
    assert np.array_equal(qx1, qx2), float(np.abs(qx1.astype(np.float64) - qx2).max())
    assert np.array_equal(qy1, qy2), float(np.abs(qy1.astype(np.float64) - qy2).max())
    for k in ("t", "dt", "step", "h_max", "V_in", "cfl_exceed"):
        assert L2[k] == L1[k], (k, L1[k], L2[k])
    scale = max(L1["V_in"], L1["volume"], 1e-300)
    for k in ("V_out", "V_clip"):
        assert abs(L2[k] - L1[k]) <= rel_sum * scale, (k, L1[k], L2[k])
    assert abs(L2["volume"] - L1["volume"]) <= rel_vol * scale


def pair(p, steps, precision, kernel, k, n_parts, halo):
    Fm = F()
    single = run(Fm.Sim(p, precision=precision, kernel=kernel, steps_per_launch=k), steps)
    dec = run(Fm.Decomp(p, n_parts, halo, precision=precision, kernel=kernel, steps_per_launch=k), steps)
    return single, dec


# ---------------------------------------------------------------- 128^2 channel, FP64, 1000 steps
@pytest.mark.parametrize("n_parts,halo", [(2, 1), (2, 4), (4, 4), (3, 16)])
def test_c1_fp64_parts_equal_single_grid_1000_steps(n_parts, halo):
    p = inputs.c1_tilted_channel()
    single, dec = pair(p, 1000, F().F64, 1, 0, n_parts, halo)
    assert single[1]["V_out"] > 0 and single[1]["V_in"] > 0
    compare(single, dec, 1e-12)


# ---------------------------------------------------------------- 2048^2 fractal, FP32, 1000 steps
@pytest.fixture(scope="module")
def c2_wet():
    p = inputs.c2_fractal()
    p.h0 = inputs.wet_start(p.z, p.dx, 0.3)
    return as_f32(p)


@pytest.mark.parametrize("kernel,k,n_parts,halo", [(3, 4, 2, 4), (3, 4, 4, 4), (3, 4, 4, 8), (3, 2, 2, 3),
                                                   (4, 0, 2, 1), (4, 0, 4, 4), (5, 0, 4, 4), (2, 0, 2, 2)])
def test_c2_fp32_parts_equal_single_grid_1000_steps(c2_wet, kernel, k, n_parts, halo):
    single, dec = pair(c2_wet, 1000, F().F32, kernel, k, n_parts, halo)
    assert single[1]["V_out"] > 0
    compare(single, dec, 1e-6)


def test_c2_fp32_auto_kernel_parts_equal_single_grid(c2_wet):
    """The default (AUTO: temporal blocking, 4 steps per launch) with a halo of 4 rows."""
    single, dec = pair(c2_wet, 256, F().F32, 0, 0, 4, 4)
    compare(single, dec, 1e-6)


# ---------------------------------------------------------------- scheme options, ragged shapes, every boundary kind
@pytest.mark.parametrize("theta,friction", [(1.0, 1), (0.8, 0), (0.9, 1)])
@pytest.mark.parametrize("precision,kernel", [(1, 1), (0, 4), (0, 5), (0, 1)])
def test_options_parts_equal_single_grid(theta, friction, precision, kernel):
    p = inputs.random_small(71, 45, 11)
    p.opts = dataclasses.replace(p.opts, theta=theta, friction=friction)
    q = p if precision == 1 else as_f32(p)
    single, dec = pair(q, 120, precision, kernel, 0, 3, 4)
    compare(single, dec, 1e-12 if precision == 1 else 1e-6)


@pytest.mark.parametrize("shape,seed,n_parts,halo", [((33, 17), 0, 3, 4), ((40, 8), 1, 2, 4), ((1, 40), 3, 4, 2),
                                                     ((257, 129), 6, 4, 3), ((129, 33), 9, 1, 4),
                                                     ((64, 64), 2, 8, 8)])
@pytest.mark.parametrize("precision,kernel,k", [(1, 1, 0), (0, 3, 4), (0, 4, 0)])
def test_ragged_parts_equal_single_grid(shape, seed, n_parts, halo, precision, kernel, k):
    """Sections crossing the cuts (inflow on xmin and ymax, outflow on xmax and
    ymin), strips as thin as the halo, one-column grids, a single part."""
    p = inputs.random_small(shape[0], shape[1], seed)
    q = p if precision == 1 else as_f32(p)
    single, dec = pair(q, 100, precision, kernel, k, n_parts, halo)
    compare(single, dec, 1e-12 if precision == 1 else 1e-6)


# ---------------------------------------------------------------- the parts themselves
def test_parts_own_rows_and_ledgers_add_up():
    Fm = F()
    p = inputs.random_small(50, 41, 4)
    d = Fm.Decomp(p, 3, 4, precision=Fm.F64)
    d.step(40)
    rows, _ = Fm.flood_decomp_plan(p.ny, 3, 4)
    h = d.read(Fm.FIELD_H)
    parts = [d.part_ledger(k) for k in range(3)]
    assert parts[1][2] == 0.0 and parts[2][2] == 0.0      # only part 0 books the inflow volume
    whole = np.array([d.ledger()[k] for k in Fm.LEDGER_KEYS])
    assert np.array_equal(Fm.flood_decomp_combine_ledgers(np.array(parts)), whole)
    for k, (y0, y1, a, b) in enumerate(rows):
        view = d.part_view(k)                             # the part's stored rows
        assert view.ny == b - a
        assert np.array_equal(view.read(Fm.FIELD_H)[y0 - a:y1 - a], h[y0:y1])
        with pytest.raises(Fm.FloodError) as e:            # parts are stepped by their decomposition
            view.step(1)
        assert e.value.status == Fm.ERR_STATE
        view.close()
    d.close()


def test_write_state_reaches_every_part_and_halo():
    Fm = F()
    p = inputs.random_small(37, 29, 5)
    rng = np.random.default_rng(3)
    h = p.h0 + rng.uniform(0, 0.05, (p.ny, p.nx))
    qx = rng.uniform(-0.01, 0.01, (p.ny, p.nx + 1))
    qy = rng.uniform(-0.01, 0.01, (p.ny + 1, p.nx))
    qx[:, 0] = qx[:, -1] = 0
    qy[0] = qy[-1] = 0
    d = Fm.Decomp(p, 4, 2, precision=Fm.F64)
    d.write_state(h, qx, qy)
    assert np.array_equal(d.read(Fm.FIELD_H), h)
    assert np.array_equal(d.read(Fm.FIELD_QX), qx)
    assert np.array_equal(d.read(Fm.FIELD_QY), qy)
    # the halo rows too: continuing equals a single grid started from the same state
    d.step(30)
    s = Fm.Sim(p, precision=Fm.F64)
    s.write_state(h, qx, qy)
    s.step(30)
    assert np.array_equal(d.read(Fm.FIELD_H), s.read(Fm.FIELD_H))
    d.close()
    s.close()


def test_decomp_rejects_strips_thinner_than_the_halo():
    Fm = F()
    p = inputs.random_small(20, 10, 1)
    with pytest.raises(Fm.FloodError) as e:
        Fm.Decomp(p, 4, 3, precision=Fm.F64)
    assert e.value.status == Fm.ERR_ARG
