"""GPU forward step vs the FP64 oracle, through the C ABI.

Tolerances (written here, derived from the arithmetic): the FP64 GPU path
evaluates every operation IEEE-rounded in the oracle's order, so it differs
only by CUDA's cbrt/pow versus the C library's (about 1 ulp) and by the order
of the Eq. 6 and ledger sums; 1e-10 m after 1000 steps.  The FP32 path
carries a relative rounding of about 6e-8 per operation on water levels of
10-100 m (a few micrometres per step) and may flip wet/dry decisions at
fronts; 1e-3 m max-abs depth and 1e-5 relative volume after 1000 steps.
Both sides get the same inputs: for FP32 the oracle runs on the float32
rounding of the DEM, roughness and initial state.
"""
import numpy as np
import pytest

import inputs
from inputs import INFLOW, OUTFLOW, XMAX, XMIN, YMAX, YMIN, Options, Problem, Section
import oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32_H = 1e-3
TOL32_MASS = 1e-5


def F():
    import paper_2204_10323_gb300 as F
    return F


def as_f32_problem(p):
    """Same problem with every grid input rounded to float32 (then held as float64)."""
    r = lambda a: None if a is None else a.astype(np.float32).astype(np.float64)
    return Problem(p.name, p.nx, p.ny, p.dx, r(p.z), r(p.n), p.sections, p.opts, h0=r(p.h0), qx0=r(p.qx0),
                   qy0=r(p.qy0), steps=p.steps, gauges=p.gauges)


def run_pair(p, steps, precision, kernel=0, **kw):
    Fm = F()
    q = as_f32_problem(p) if precision == Fm.F32 else p
    o = oracle.Oracle(q)
    V0 = o.volume()
    o.run(steps)
    s = Fm.Sim(q, precision=precision, kernel=kernel, **kw)
    s.step(steps)
    s.sync()
    h, qx, qy = s.state()
    L = s.ledger()
    s.close()
    return o, V0, h.astype(np.float64), qx.astype(np.float64), qy.astype(np.float64), L


def check_ledger(o, L, rel):
    Lo = o.ledger_dict()
    scale = max(Lo["V_in"], o.volume(), 1e-300)
    for k in ("V_in", "V_out", "V_clip"):
        assert abs(L[k] - Lo[k]) <= rel * scale, (k, L[k], Lo[k])
    assert abs(L["volume"] - o.volume()) <= rel * scale
    assert L["t"] == pytest.approx(Lo["t"], rel=1e-12)
    assert L["step"] == Lo["step"]


# ---------------------------------------------------------------- FP64 parity
def test_c1_fp64_matches_oracle_1000_steps():
    p = inputs.c1_tilted_channel()
    o, V0, h, qx, qy, L = run_pair(p, 1000, F().F64)
    assert np.abs(h - o.h).max() < TOL64
    assert np.abs(qx - o.qx).max() < TOL64
    assert np.abs(qy - o.qy).max() < TOL64
    check_ledger(o, L, 1e-12)


@pytest.mark.parametrize("shape,seed", [((33, 17), 0), ((7, 5), 1), ((130, 70), 2), ((1, 9), 3), ((9, 1), 4)])
def test_random_fp64_matches_oracle(shape, seed):
    p = inputs.random_small(shape[0], shape[1], seed)
    o, V0, h, qx, qy, L = run_pair(p, 120, F().F64)
    assert np.abs(h - o.h).max() < TOL64
    assert np.abs(qx - o.qx).max() < TOL64
    assert np.abs(qy - o.qy).max() < TOL64
    check_ledger(o, L, 1e-12)


@pytest.mark.parametrize("bc_form,dt_mode", [(1, 0), (0, 1), (1, 1)])
def test_options_fp64_match_oracle(bc_form, dt_mode):
    p = inputs.random_small(40, 23, 5, bc_form=bc_form, dt_mode=dt_mode)
    o, V0, h, qx, qy, L = run_pair(p, 80, F().F64)
    assert np.abs(h - o.h).max() < TOL64
    check_ledger(o, L, 1e-12)


# ---------------------------------------------------------------- FP32 parity
@pytest.mark.parametrize("kernel", [1, 2, 4, 5])
def test_c1_fp32_matches_oracle_1000_steps(kernel):
    p = inputs.c1_tilted_channel()
    o, V0, h, qx, qy, L = run_pair(p, 1000, F().F32, kernel=kernel)
    assert np.abs(h - o.h).max() < TOL32_H
    Vo = o.volume()
    assert abs(L["volume"] - Vo) / Vo < TOL32_MASS
    # the FP32 run's own ledger closes too
    bal = L["volume"] - V0 - (L["V_in"] - L["V_out"] + L["V_clip"])
    assert abs(bal) / L["V_in"] < TOL32_MASS


@pytest.mark.parametrize("kernel", [1, 2, 4, 5])
@pytest.mark.parametrize("shape,seed", [((33, 17), 0), ((7, 5), 1), ((130, 70), 2), ((257, 129), 6),
                                        ((1, 1), 7), ((1, 40), 3), ((40, 1), 4), ((128, 32), 8), ((129, 33), 9)])
def test_random_fp32_matches_oracle(kernel, shape, seed):
    p = inputs.random_small(shape[0], shape[1], seed)
    o, V0, h, qx, qy, L = run_pair(p, 100, F().F32, kernel=kernel)
    assert np.abs(h - o.h).max() < TOL32_H
    assert np.abs(qx - o.qx).max() < 10 * TOL32_H
    assert np.abs(qy - o.qy).max() < 10 * TOL32_H


@pytest.mark.parametrize("kernel,k", [(1, 0), (2, 0), (4, 0), (5, 0), (3, 4)])
def test_literal_bc_form_fp32_matches_oracle(kernel, k):
    """Eq. 5 taken literally (A = dx^2, dx^2 h^(2/3) sqrt(S)/n) on every FP32 kernel family."""
    p = inputs.random_small(97, 61, 23, bc_form=1)
    o, V0, h, qx, qy, L = run_pair(p, 200, F().F32, kernel=kernel, steps_per_launch=k)
    assert np.abs(h - o.h).max() < TOL32_H
    assert abs(L["V_out"] - o.ledger.V_out) <= 1e-5 * max(o.ledger.V_out, 1.0)


def test_c2_fp32_parity_1000_steps():
    """The 2048^2 fractal workload at reduced size (256^2 crop of the same generator)."""
    p = inputs.c2_fractal(nx=256, ny=256, steps=1000)
    o, V0, h, qx, qy, L = run_pair(p, 1000, F().F32)
    assert np.abs(h - o.h).max() < TOL32_H
    Vo = o.volume()
    assert abs(L["volume"] - Vo) / max(Vo, 1.0) < TOL32_MASS


# ---------------------------------------------------------------- invariants on the GPU
@pytest.mark.parametrize("precision,kernel", [(0, 1), (0, 2), (0, 4), (0, 5), (1, 1)])
def test_lake_at_rest_is_exact_on_gpu(precision, kernel):
    p = inputs.lake_at_rest(67, 45)
    s = F().Sim(p, precision=precision, kernel=kernel)
    h0 = s.read(F().FIELD_H).copy()
    s.step(300)
    h, qx, qy = s.state()
    assert np.array_equal(h, h0)
    assert not qx.any() and not qy.any()


def test_fp32_run_is_deterministic_and_resumable():
    Fm = F()
    p = as_f32_problem(inputs.random_small(150, 90, 11))
    a = Fm.Sim(p)
    a.step(100)
    ha, qxa, qya = a.state()
    b = Fm.Sim(p)
    b.step(37)                         # mid-epoch stop (E = 4)
    hb, qxb, qyb = b.state()
    Lb = b.ledger()
    c = Fm.Sim(p)
    c.write_state(hb, qxb, qyb)
    c.set_clock(Lb["t"], int(Lb["step"]), Lb["dt"], Lb["V_in"], Lb["V_out"], Lb["V_clip"])
    c.step(63)
    hc, qxc, qyc = c.state()
    a2 = Fm.Sim(p)
    a2.step(100)
    assert np.array_equal(ha, a2.read(Fm.FIELD_H))
    assert np.array_equal(ha, hc) and np.array_equal(qxa, qxc) and np.array_equal(qya, qyc)


@pytest.mark.parametrize("use_graph", [0, 1])
def test_write_state_mid_run_swaps_halves_under_graph_replay(use_graph):
    # write_state makes the staged half current (the halves swap); captured
    # epochs are kept per half, so replay continues from the written state
    Fm = F()
    p = as_f32_problem(inputs.random_small(150, 90, 12))
    p.opts.epoch_steps = 4
    a = Fm.Sim(p, use_graph=use_graph)
    a.step(12)
    h1, qx1, qy1 = a.state()
    L1 = a.ledger()
    a.step(5)                            # move on, then rewind to the saved state
    for k in range(3):                   # both halves current in turn
        a.write_state(h1, qx1, qy1)
        a.set_clock(L1["t"], int(L1["step"]), L1["dt"], L1["V_in"], L1["V_out"], L1["V_clip"])
        a.step(k + 1)
    a.write_state(h1, qx1, qy1)
    a.set_clock(L1["t"], int(L1["step"]), L1["dt"], L1["V_in"], L1["V_out"], L1["V_clip"])
    a.step(20)
    b = Fm.Sim(p)
    b.step(32)
    for f in (Fm.FIELD_H, Fm.FIELD_QX, Fm.FIELD_QY):
        assert np.array_equal(a.read(f), b.read(f)), f
    a.close()
    b.close()


def test_write_state_of_an_ensemble_member():
    Fm = F()
    probs = [as_f32_problem(inputs.random_small(nx, ny, 20 + k)) for k, (nx, ny) in enumerate([(150, 90), (64, 40)])]
    for q in probs:
        q.opts.epoch_steps = 4
    ref = Fm.Sim(probs[1])
    ref.step(8)
    h8, qx8, qy8 = ref.state()
    L8 = ref.ledger()
    ref.step(8)
    e = Fm.Ensemble(probs)
    e.step(4)
    m = e.members[1]
    m.write_state(h8, qx8, qy8)
    m.set_clock(L8["t"], 4, L8["dt"], L8["V_in"], L8["V_out"], L8["V_clip"])
    e.step(8)
    assert np.array_equal(m.read(Fm.FIELD_H), ref.read(Fm.FIELD_H))
    e.close()
    ref.close()


def test_inflow_distribution_matches_oracle_eq6():
    """First-step boundary faces equal the oracle's Eq. 6 split (FP64)."""
    Fm = F()
    p = inputs.random_small(30, 24, 4)
    o = oracle.Oracle(p)
    s = Fm.Sim(p, precision=Fm.F64)
    s.step(1)
    qx = s.read(Fm.FIELD_QX)
    a, b = o.section_range(0)
    W, q = o.inflow_faces(0, o.hydrograph(0, 0.0))
    np.testing.assert_allclose(qx[a:b, 0], q, rtol=1e-12, atol=1e-15)


def test_graph_replay_equals_direct_launches():
    Fm = F()
    p = as_f32_problem(inputs.random_small(200, 120, 12))
    a = Fm.Sim(p)
    a.step(64)
    b = Fm.Sim(p, use_graph=True)
    b.step(10)
    b.step(54)
    assert np.array_equal(a.read(Fm.FIELD_H), b.read(Fm.FIELD_H))
    assert np.array_equal(a.read(Fm.FIELD_QX), b.read(Fm.FIELD_QX))


def test_gauge_series_matches_state_reads():
    Fm = F()
    p = as_f32_problem(inputs.random_small(60, 40, 13))
    g = np.array([[3, 4], [59, 39], [0, 0], [30, 20]])
    a = Fm.Sim(p)
    series = a.run_gauges(9, g)
    b = Fm.Sim(p)
    for k in range(9):
        b.step(1)
        h = b.read(Fm.FIELD_H)
        np.testing.assert_array_equal(series[k], h[g[:, 1], g[:, 0]].astype(np.float64))


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """A device wait on an mbarrier nothing arrives at gives up after its budget
    (the path a lost copy takes in every step kernel) and reports a timeout;
    the context then runs a simulation as before."""
    import time
    Fm = F()
    t0 = time.perf_counter()
    assert Fm.lib().flood_check_bounded_wait(0.002) == Fm.ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert "gave up" in Fm.flood_last_error(None)
    p = as_f32_problem(inputs.random_small(33, 17, 0))
    o, V0, h, qx, qy, L = run_pair(p, 20, Fm.F32)
    assert np.abs(h - o.h).max() < TOL32_H


def test_nonfinite_depth_is_reported_and_sticky():
    Fm = F()
    p = inputs.random_small(20, 12, 2)
    s = Fm.Sim(p)
    h = s.read(Fm.FIELD_H)
    h[3, 4] = np.inf
    # write_state rejects non-finite host input
    with pytest.raises(Fm.FloodError):
        s.write_state(h)
    import torch
    hd = torch.from_numpy(h).cuda()          # device input is not scanned on the host
    s.write_state(hd)
    s.step(8)
    with pytest.raises(Fm.FloodError) as e:
        s.sync()
    assert e.value.status == Fm.ERR_NONFINITE
    with pytest.raises(Fm.FloodError) as e:
        s.step(1)
    assert e.value.status == Fm.ERR_STATE
    s.write_state(np.zeros_like(h))          # clears the error
    s.step(4)
    s.sync()


@pytest.mark.parametrize("precision,kernel", [(0, 0), (0, 4), (1, 1)])
def test_broken_courant_limit_is_reported_and_sticky(precision, kernel):
    """A constant time step far above the Courant limit: 5 s on 1 m cells with
    depths up to 2 m gives dt sqrt(g h) = 22 > dx.  The lake stays at rest
    (Eq. 3 gives q = 0 on a flat water surface), so the status is the only report."""
    import dataclasses
    Fm = F()
    p = inputs.lake_at_rest(16, 12)
    p.opts = dataclasses.replace(p.opts, dt_const=5.0)
    E = p.opts.epoch_steps
    s = Fm.Sim(p, precision=precision, kernel=kernel)
    h0 = s.read(Fm.FIELD_H).copy()
    s.step(E)                                # the first epoch start has no earlier epoch to check
    s.sync()
    s.step(1)                                # the second epoch start checks the first epoch
    with pytest.raises(Fm.FloodError) as e:
        s.sync()
    assert e.value.status == Fm.ERR_CFL
    L = s.ledger()
    assert L["cfl_exceed"] == 1 and L["step"] == E + 1
    assert np.array_equal(s.read(Fm.FIELD_H), h0)
    with pytest.raises(Fm.FloodError) as e:
        s.step(1)
    assert e.value.status == Fm.ERR_STATE
    s.write_state(h0)                        # clears the error
    s.step(4)                                # inside the epoch: no new check
    s.sync()
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_depth_clip_matches_oracle(precision):
    """Thin water drained through two outflow edges goes negative and is clipped."""
    Fm = F()
    z = np.zeros((6, 8))
    secs = [Section.cells(XMAX, 0, 6, OUTFLOW, 0.5, 8, 6), Section.cells(YMIN, 0, 8, OUTFLOW, 0.5, 8, 6)]
    p = Problem("clip", 8, 6, 0.1, z, np.full((6, 8), 0.01), secs, Options(dt_mode=1, dt_const=0.05),
                h0=np.full((6, 8), 0.002))
    o, V0, h, qx, qy, L = run_pair(p, 20, precision, kernel=2 if precision == 0 else 1)
    assert o.ledger.V_clip > 0
    tol = TOL64 if precision == 1 else 1e-6
    assert np.abs(h - o.h).max() < tol
    assert L["V_clip"] == pytest.approx(o.ledger.V_clip, rel=1e-12 if precision == 1 else 1e-4)


def test_empty_section_and_zero_inflow():
    Fm = F()
    nx, ny = 20, 10
    z = np.zeros((ny, nx))
    secs = [Section(XMIN, 0.3, 0.3, INFLOW, 1e-3, np.array([0.0, 1.0]), np.array([5.0, 5.0])),
            Section.cells(YMAX, 2, 9, INFLOW, 1e-3, nx, ny, [0.0, 1.0], [0.0, 0.0]),
            Section.cells(XMAX, 0, ny, OUTFLOW, 1e-3, nx, ny)]
    p = Problem("empty", nx, ny, 1.0, z, np.full((ny, nx), 0.03), secs, Options(dt_mode=1), h0=np.full((ny, nx), 0.1))
    o = oracle.Oracle(p)
    o.run(20)
    s = Fm.Sim(p, precision=Fm.F64)
    s.step(20)
    assert np.abs(s.read(Fm.FIELD_H) - o.h).max() < TOL64
    assert s.ledger()["V_in"] == 0.0


# ---------------------------------------------------------------- theta-weighted faces
def with_theta(p, theta):
    p.opts.theta = theta
    return p


@pytest.mark.parametrize("theta", [0.9, 0.7])
@pytest.mark.parametrize("shape,seed", [((33, 17), 0), ((130, 70), 2), ((1, 9), 3), ((9, 1), 4)])
def test_theta_fp64_matches_oracle(theta, shape, seed):
    p = with_theta(inputs.random_small(shape[0], shape[1], seed), theta)
    o, V0, h, qx, qy, L = run_pair(p, 120, F().F64)
    assert np.abs(h - o.h).max() < TOL64
    assert np.abs(qx - o.qx).max() < TOL64
    assert np.abs(qy - o.qy).max() < TOL64
    check_ledger(o, L, 1e-12)


def test_theta_fp64_channel_1000_steps():
    # theta = 0.8: at theta = 0.7 the channel at the CFL limit (alpha 0.7, 2 s steps)
    # diverges after ~750 steps in the oracle as on the GPU (a property of the scheme)
    p = with_theta(inputs.c1_tilted_channel(), 0.8)
    o, V0, h, qx, qy, L = run_pair(p, 1000, F().F64)
    assert np.abs(h - o.h).max() < TOL64
    check_ledger(o, L, 1e-12)


@pytest.mark.parametrize("kernel", [1, 4, 5, 3])
@pytest.mark.parametrize("shape,seed", [((130, 70), 2), ((257, 129), 6), ((129, 33), 9)])
def test_theta_fp32_matches_oracle(kernel, shape, seed):
    p = with_theta(inputs.random_small(shape[0], shape[1], seed), 0.8)
    o, V0, h, qx, qy, L = run_pair(p, 100, F().F32, kernel=kernel)
    assert np.abs(h - o.h).max() < TOL32_H
    assert np.abs(qx - o.qx).max() < 10 * TOL32_H
    assert np.abs(qy - o.qy).max() < 10 * TOL32_H


@pytest.mark.parametrize("tile", [(0, 0), (2, 9), (1, 3)])
def test_theta_tma_tiles_equal_row_staging_bitwise(tile):
    Fm = F()
    p = as_f32_problem(with_theta(inputs.random_small(257, 129, 6), 0.75))
    a = Fm.Sim(p, kernel=Fm.KERNEL_STREAM, tile=tile)
    b = Fm.Sim(p, kernel=Fm.KERNEL_TMA, tile=tile)
    a.step(37)
    b.step(37)
    for f in (Fm.FIELD_H, Fm.FIELD_QX, Fm.FIELD_QY):
        assert np.array_equal(a.read(f), b.read(f)), f


@pytest.mark.parametrize("theta,friction", [(0.75, 0), (1.0, 1), (0.75, 1)])
@pytest.mark.parametrize("K,E,tile", [(4, 4, (0, 0)), (4, 8, (2, 9)), (2, 4, (1, 3)), (3, 6, (3, 40)),
                                      (1, 4, (0, 0)), (8, 8, (0, 0)), (8, 16, (2, 17))])
def test_options_temporal_blocking_equals_single_steps_bitwise(theta, friction, K, E, tile):
    """K steps per launch with the theta weighting and/or the vector norm give the
    bits of K single steps of the stream kernel (the same face arithmetic), on
    ragged grids with several strips, chunk seams and pipelines walking many items."""
    Fm = F()
    for shape, seed in (((257, 129), 6), ((130, 70), 2), ((33, 17), 0)):
        p = as_f32_problem(with_friction(inputs.random_small(shape[0], shape[1], seed), friction, theta))
        p.opts.epoch_steps = E
        a = Fm.Sim(p, kernel=Fm.KERNEL_STREAM)
        b = Fm.Sim(p, kernel=Fm.KERNEL_TILED, steps_per_launch=K, tile=tile)
        for n in (3 * E, 5, 2 * E + 1):
            a.step(n)
            b.step(n)
        for f in (Fm.FIELD_H, Fm.FIELD_QX, Fm.FIELD_QY):
            assert np.array_equal(a.read(f), b.read(f)), (shape, f)
        La, Lb = a.ledger(), b.ledger()
        for k in ("t", "dt", "V_in", "volume", "h_max", "step"):
            assert La[k] == pytest.approx(Lb[k], rel=1e-12, abs=1e-12), k
        for k in ("V_out", "V_clip"):
            assert La[k] == pytest.approx(Lb[k], rel=1e-6, abs=1e-9), k
        a.close()
        b.close()


@pytest.mark.parametrize("kernel,K", [(4, 0), (3, 4), (3, 2)])
@pytest.mark.parametrize("theta,friction", [(0.8, 0), (1.0, 1), (0.8, 1)])
def test_options_ensemble_members_equal_solo_runs(kernel, K, theta, friction):
    Fm = F()
    probs = []
    for nx, ny, seed in ((130, 70, 2), (257, 129, 6), (64, 300, 17), (33, 17, 0)):
        probs.append(as_f32_problem(with_friction(inputs.random_small(nx, ny, seed), friction, theta)))
    ens = Fm.Ensemble(probs)
    E = probs[0].opts.epoch_steps
    ens.set_launch(2, 16, 2 * E)
    ens.set_kernel(kernel, K)
    ens.step(3)
    ens.step(4 * E)
    n = 3 + 4 * E
    for mb, p in zip(ens.members, probs):
        s = Fm.Sim(p, kernel=Fm.KERNEL_STREAM)
        s.step(n)
        for f in (Fm.FIELD_H, Fm.FIELD_QX, Fm.FIELD_QY):
            assert np.array_equal(mb.read(f), s.read(f)), (p.name, f)
        s.close()
    ens.close()


# ---------------------------------------------------------------- vector-norm friction
def with_friction(p, friction, theta=1.0):
    p.opts.friction = friction
    p.opts.theta = theta
    return p


def test_vector_friction_changes_the_solution():
    # the parity cases below see the term: on these inputs the two readings of
    # |q| differ by far more than the FP32 tolerance
    a = oracle.Oracle(inputs.random_small(257, 129, 6))
    b = oracle.Oracle(with_friction(inputs.random_small(257, 129, 6), 1))
    a.run(100)
    b.run(100)
    assert np.abs(a.h - b.h).max() > 30 * TOL32_H


@pytest.mark.parametrize("theta", [1.0, 0.8])
@pytest.mark.parametrize("shape,seed", [((33, 17), 0), ((130, 70), 2), ((1, 9), 3), ((9, 1), 4)])
def test_vector_friction_fp64_matches_oracle(theta, shape, seed):
    p = with_friction(inputs.random_small(shape[0], shape[1], seed), 1, theta)
    o, V0, h, qx, qy, L = run_pair(p, 120, F().F64)
    assert np.abs(h - o.h).max() < TOL64
    assert np.abs(qx - o.qx).max() < TOL64
    assert np.abs(qy - o.qy).max() < TOL64
    check_ledger(o, L, 1e-12)


def test_vector_friction_fp64_channel_1000_steps():
    p = with_friction(inputs.c1_tilted_channel(), 1)
    o, V0, h, qx, qy, L = run_pair(p, 1000, F().F64)
    assert np.abs(h - o.h).max() < TOL64
    check_ledger(o, L, 1e-12)


@pytest.mark.parametrize("kernel", [1, 4, 5, 3])
@pytest.mark.parametrize("theta", [1.0, 0.8])
@pytest.mark.parametrize("shape,seed", [((130, 70), 2), ((257, 129), 6), ((129, 33), 9)])
def test_vector_friction_fp32_matches_oracle(kernel, theta, shape, seed):
    p = with_friction(inputs.random_small(shape[0], shape[1], seed), 1, theta)
    o, V0, h, qx, qy, L = run_pair(p, 100, F().F32, kernel=kernel)
    assert np.abs(h - o.h).max() < TOL32_H
    assert np.abs(qx - o.qx).max() < 10 * TOL32_H
    assert np.abs(qy - o.qy).max() < 10 * TOL32_H
    check_ledger(o, L, TOL32_MASS)


@pytest.mark.parametrize("kernel", [4, 5, 3])
def test_vector_friction_fp32_channel_1000_steps(kernel):
    p = with_friction(inputs.c1_tilted_channel(), 1)
    o, V0, h, qx, qy, L = run_pair(p, 1000, F().F32, kernel=kernel)
    assert np.abs(h - o.h).max() < TOL32_H
    assert abs(L["volume"] - o.volume()) <= TOL32_MASS * o.volume()


@pytest.mark.parametrize("theta", [1.0, 0.75])
@pytest.mark.parametrize("tile", [(0, 0), (2, 9), (1, 3)])
def test_vector_friction_tma_tiles_equal_row_staging_bitwise(theta, tile):
    Fm = F()
    p = as_f32_problem(with_friction(inputs.random_small(257, 129, 6), 1, theta))
    a = Fm.Sim(p, kernel=Fm.KERNEL_STREAM, tile=tile)
    b = Fm.Sim(p, kernel=Fm.KERNEL_TMA, tile=tile)
    a.step(37)
    b.step(37)
    for f in (Fm.FIELD_H, Fm.FIELD_QX, Fm.FIELD_QY):
        assert np.array_equal(a.read(f), b.read(f)), f


def test_vector_friction_auto_equals_the_tensor_tile_kernel():
    """AUTO runs the options on the temporal-blocking kernel (E = 16 is a multiple
    of 4); its bits are the TMA-tile kernel's."""
    Fm = F()
    p = as_f32_problem(with_friction(inputs.random_small(257, 129, 6), 1))
    a = Fm.Sim(p, kernel=Fm.KERNEL_AUTO)
    b = Fm.Sim(p, kernel=Fm.KERNEL_TMA)
    a.step(21)
    b.step(21)
    for f in (Fm.FIELD_H, Fm.FIELD_QX, Fm.FIELD_QY):
        assert np.array_equal(a.read(f), b.read(f)), f


# ---------------------------------------------------------------- coarsening
def block_mean(a, f):
    """Mean over f x f blocks (partial blocks at the far edges over their cells), in float64."""
    ny, nx = a.shape
    out = np.empty((-(-ny // f), -(-nx // f)))
    for J in range(out.shape[0]):
        for I in range(out.shape[1]):
            out[J, I] = a[J * f:(J + 1) * f, I * f:(I + 1) * f].astype(np.float64).mean()
    return out


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("shape,f", [((64, 48), 2), ((37, 29), 4), ((5, 3), 8), ((16, 16), 1), ((1, 9), 2)])
def test_coarsen_matches_block_mean(dtype, shape, f):
    import torch
    Fm = F()
    z = np.random.default_rng(5).normal(10.0, 3.0, size=shape).astype(dtype)
    ref = block_mean(z, f).astype(dtype)
    rtol = 1e-15 if dtype == np.float64 else 1.2e-7
    np.testing.assert_allclose(Fm.coarsen(z, f), ref, rtol=rtol)
    zd = torch.from_numpy(z).cuda()
    np.testing.assert_allclose(Fm.coarsen(zd, f).cpu().numpy(), ref, rtol=rtol)


# ---------------------------------------------------------------- final-step truncation
def _advance_pair(p, precision, targets, kernel=0, k=0):
    """Oracle and GPU through the same sequence of advances and whole steps."""
    Fm = F()
    q = as_f32_problem(p) if precision == Fm.F32 else p
    o = oracle.Oracle(q)
    s = Fm.Sim(q, precision=precision, kernel=kernel, steps_per_launch=k)
    for T in targets:
        if isinstance(T, int):               # whole steps
            o.run(T)
            s.step(T)
        else:
            na, nb = s.advance(T), o.advance(T)
            # FP32 picks its CFL dt from an FP32 depth maximum: a target within
            # rounding of a step end may split differently, so only FP64 counts
            if precision == Fm.F64:
                assert na == nb
            assert s.ledger()["t"] == T == o.ledger.t
    return o, s


def test_advance_fp64_matches_oracle():
    p = inputs.random_small(70, 45, 21)
    o, s = _advance_pair(p, F().F64, [0.37, 3, 1.234, 1.2341, 5, 9.9, 9.9])
    h, qx, qy = s.state()
    assert np.abs(h - o.h).max() < TOL64
    assert np.abs(qx - o.qx).max() < TOL64
    check_ledger(o, s.ledger(), 1e-12)
    assert s.ledger()["dt"] == o.ledger.dt


@pytest.mark.parametrize("kernel,k", [(4, 0), (5, 0), (3, 4)])
def test_advance_fp32_matches_oracle(kernel, k):
    p = inputs.random_small(130, 70, 22)
    o, s = _advance_pair(p, F().F32, [0.91, 7, 2.5, 2.500001, 13, 6.75], kernel=kernel, k=k)
    assert np.abs(s.read(F().FIELD_H).astype(np.float64) - o.h).max() < TOL32_H
    assert s.ledger()["V_in"] == pytest.approx(o.ledger.V_in, rel=1e-6)


def test_advance_books_the_truncated_inflow_exactly():
    """Constant Q into a closed basin: after advancing to T, V_in = Q T and the
    stored volume grew by V_in + V_clip (FP64 path)."""
    Fm = F()
    sec = Section.cells(XMIN, 1, 3, INFLOW, 1e-3, 6, 4, [0.0, 100.0], [2.0, 2.0])
    p = Problem("basin", 6, 4, 1.0, np.zeros((4, 6)), np.full((4, 6), 0.03), [sec],
                Options(dt_mode=1, dt_const=0.1), h0=np.full((4, 6), 0.5))
    s = Fm.Sim(p, precision=Fm.F64)
    V0 = s.ledger()["volume"]
    assert s.advance(0.55) == 6
    L = s.ledger()
    assert L["t"] == 0.55 and L["dt"] == 0.1
    assert L["V_in"] == pytest.approx(2.0 * 0.55, rel=1e-14)
    assert L["volume"] - V0 == pytest.approx(L["V_in"] + L["V_clip"], rel=1e-12)
    with pytest.raises(Fm.FloodError):
        s.advance(0.5)


# ---------------------------------------------------------------- temporal blocking
@pytest.mark.parametrize("K", [1, 2, 3, 4, 8])
@pytest.mark.parametrize("shape,seed", [((130, 70), 2), ((257, 129), 6), ((241, 50), 14), ((120, 33), 15),
                                        ((7, 5), 1), ((1, 40), 3), ((40, 1), 4), ((361, 97), 16)])
def test_tiled_equals_single_steps_bitwise(K, shape, seed):
    """K time levels per launch give the same bits and ledger as K single steps."""
    Fm = F()
    p = as_f32_problem(inputs.random_small(shape[0], shape[1], seed))
    p.opts.epoch_steps = {1: 4, 2: 4, 3: 3, 4: 4, 8: 8}[K]
    a = Fm.Sim(p, kernel=Fm.KERNEL_STREAM)
    b = Fm.Sim(p, kernel=Fm.KERNEL_TILED, steps_per_launch=K)
    for n in (5, 12, 1, 30):              # stops inside and at the ends of epochs
        a.step(n)
        b.step(n)
    for f in (Fm.FIELD_H, Fm.FIELD_QX, Fm.FIELD_QY):
        assert np.array_equal(a.read(f), b.read(f)), f
    La, Lb = a.ledger(), b.ledger()
    for k in ("V_in", "volume", "t", "h_max"):
        assert Lb[k] == pytest.approx(La[k], rel=1e-12, abs=1e-12), k
    # the tiled kernel sums boundary outflow and clipped depth per lane in float
    # over runs of at most 32 rows before folding them into the double ledger
    for k in ("V_out", "V_clip"):
        assert Lb[k] == pytest.approx(La[k], rel=1e-6, abs=1e-9), k


@pytest.mark.parametrize("K", [2, 4, 8])
@pytest.mark.parametrize("shape,seed,tile", [((361, 97), 16, (3, 16)), ((257, 129), 6, (5, 7)),
                                             ((130, 70), 2, (1, 9)), ((40, 33), 4, (2, 1))])
def test_tiled_many_items_per_pipeline_bitwise(K, shape, seed, tile):
    """Few pipelines walking many (chunk, strip) items each: the staging ring
    carries its slots and phases from item to item."""
    Fm = F()
    p = as_f32_problem(inputs.random_small(shape[0], shape[1], seed))
    p.opts.epoch_steps = max(4, K)
    a = Fm.Sim(p, kernel=Fm.KERNEL_STREAM)
    b = Fm.Sim(p, kernel=Fm.KERNEL_TILED, steps_per_launch=K, tile=tile)
    for n in (5, 12, 1, 30):
        a.step(n)
        b.step(n)
    for f in (Fm.FIELD_H, Fm.FIELD_QX, Fm.FIELD_QY):
        assert np.array_equal(a.read(f), b.read(f)), f
    La, Lb = a.ledger(), b.ledger()
    for k in ("V_in", "volume", "h_max"):
        assert Lb[k] == pytest.approx(La[k], rel=1e-12, abs=1e-12), k
    for k in ("V_out", "V_clip"):
        assert Lb[k] == pytest.approx(La[k], rel=1e-6, abs=1e-9), k


@pytest.mark.parametrize("shape,seed,tile", [((130, 70), 2, (0, 0)), ((257, 129), 6, (2, 9)), ((7, 5), 1, (0, 0)),
                                             ((1, 40), 3, (1, 3)), ((40, 1), 4, (0, 0)), ((361, 97), 16, (4, 64)),
                                             ((129, 33), 9, (3, 1))])
def test_tma_tiles_equal_row_staging_bitwise(shape, seed, tile):
    """Rows staged as 2D tensor-map tiles (zero-filled outside the grid) give the
    bits and the ledger of rows staged by 1D bulk copies, for every launch shape."""
    Fm = F()
    p = as_f32_problem(inputs.random_small(shape[0], shape[1], seed))
    a = Fm.Sim(p, kernel=Fm.KERNEL_STREAM, tile=tile)
    b = Fm.Sim(p, kernel=Fm.KERNEL_TMA, tile=tile)
    for n in (5, 12, 1, 30):
        a.step(n)
        b.step(n)
    for f in (Fm.FIELD_H, Fm.FIELD_QX, Fm.FIELD_QY):
        assert np.array_equal(a.read(f), b.read(f)), f
    La, Lb = a.ledger(), b.ledger()
    for k in ("V_in", "V_out", "V_clip", "volume", "t", "h_max"):
        assert Lb[k] == pytest.approx(La[k], rel=1e-12, abs=1e-12), k


def test_tiled_c1_matches_oracle_and_lake_at_rest():
    Fm = F()
    p = inputs.c1_tilted_channel()
    o, V0, h, qx, qy, L = run_pair(p, 1000, Fm.F32, kernel=Fm.KERNEL_TILED, steps_per_launch=4)
    assert np.abs(h - o.h).max() < TOL32_H
    assert abs(L["volume"] - o.volume()) / o.volume() < TOL32_MASS
    lake = inputs.lake_at_rest(300, 170)
    s = Fm.Sim(lake, kernel=Fm.KERNEL_TILED, steps_per_launch=4)
    h0 = s.read(Fm.FIELD_H).copy()
    s.step(64)
    assert np.array_equal(s.read(Fm.FIELD_H), h0)
    assert not s.read(Fm.FIELD_QX).any() and not s.read(Fm.FIELD_QY).any()


def test_tiled_large_grid_many_chunks_bitwise():
    """A grid large enough for many strips and chunks per strip (persistent split)."""
    Fm = F()
    p = as_f32_problem(inputs.c2_fractal(nx=1100, ny=2300, steps=100))
    p.h0 = inputs.wet_start(p.z, p.dx, 0.3)
    a = Fm.Sim(p, kernel=Fm.KERNEL_STREAM)
    b = Fm.Sim(p, kernel=Fm.KERNEL_TILED, steps_per_launch=4)
    a.step(40)
    b.step(40)
    for f in (Fm.FIELD_H, Fm.FIELD_QX, Fm.FIELD_QY):
        assert np.array_equal(a.read(f), b.read(f)), f
