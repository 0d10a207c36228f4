"""Pins of the FP64 oracle against values the method and the mathematics fix.

None of these compares the oracle with itself: the expected values are hand
evaluations (40-digit decimal arithmetic of Eq. 3-5 written out by hand, the
literals below), closed forms (Manning normal depth, uniform inflow split),
exact invariants (lake at rest, mass ledger, mirror symmetry), library
routines (numpy.interp, scipy's brentq) and finite differences.
"""
import math

import numpy as np
import pytest

import inputs
from inputs import INFLOW, OUTFLOW, XMAX, XMIN, YMAX, YMIN, Options, Problem, Section
import oracle
from closed_forms import standing_wave_amplitudes, standing_wave_gradient


def closed_box(z, h0, dx=1.0, n=0.03, sections=(), **opt):
    ny, nx = z.shape
    o = dict(dt_mode=1, dt_const=0.1)
    o.update(opt)
    return Problem("case", nx, ny, dx, np.asarray(z, float), np.full((ny, nx), n), list(sections),
                   Options(**o), h0=np.asarray(h0, float))


# ---------------------------------------------------------------- P1: 2 cells
def test_p1_two_cell_hand_values():
    """Flat bed, dx = 1, dt = 0.1, n = 0.03, h = (1, 0.5), closed walls.

    Step 1: h_f = 1, q' = g dt h_f (1 - 0.5)/dx = 0.4905 (no friction at q = 0),
            h = (1 - 0.04905, 0.5 + 0.04905).
    Step 2: h_f = 0.95095, slope 0.4019,
            q' = (0.4905 + 0.981*0.95095*0.4019) / (1 + 0.981*0.0009*0.4905*0.95095^(-7/3)).
    Step 3: same with the step-2 state.  Decimal (40-digit) evaluations below.
    """
    p = closed_box(np.zeros((1, 2)), [[1.0, 0.5]])
    o = oracle.Oracle(p)
    expect = [
        (0.4905, 0.95095, 0.54905),
        (0.8650040113860357304, 0.8644495988613964270, 0.6355504011386035730),
        (1.0579812164048227008, 0.7586514772209141569, 0.7413485227790858431),
    ]
    for q, h0, h1 in expect:
        o.run(1)
        assert o.qx[0, 1] == pytest.approx(q, rel=1e-14, abs=1e-15)
        assert o.h[0, 0] == pytest.approx(h0, rel=1e-14)
        assert o.h[0, 1] == pytest.approx(h1, rel=1e-14)
        assert o.qx[0, 0] == 0.0 and o.qx[0, 2] == 0.0


# ---------------------------------------------------------------- P2: 4x4
def test_p2_four_by_four_hand_values():
    """Step in the bed: columns 0-1 at z = 0 with h = 1, columns 2-3 at z = 0.6 dry.

    Outflow (S = 1e-3) at the xmax face of row 0 (a dry cell) and at the xmin
    face of row 1 (a wet cell); walls elsewhere; dx = 1, dt = 0.1, n = 0.03.
    Step 1 by hand: faces 1|2 have h_f = max(1, 0.6) - max(0, 0.6) = 0.4 and
    q' = g dt 0.4 (1 - 0.6) = 0.15696; the wet outflow face carries
    -1^(5/3) sqrt(1e-3)/0.03 = -1.05409255338946; everything else is 0.
    Step 2 values are 40-digit decimal evaluations of the same formulas.
    """
    z = np.array([[0.0, 0.0, 0.6, 0.6]] * 4)
    h0 = np.array([[1.0, 1.0, 0.0, 0.0]] * 4)
    secs = [Section.cells(XMAX, 0, 1, OUTFLOW, 1e-3, 4, 4), Section.cells(XMIN, 1, 2, OUTFLOW, 1e-3, 4, 4)]
    o = oracle.Oracle(closed_box(z, h0, sections=secs))
    o.run(1)
    h1 = np.array([[1.0, 0.984304, 0.015696, 0.0],
                   [0.8945907446610540, 0.984304, 0.015696, 0.0],
                   [1.0, 0.984304, 0.015696, 0.0],
                   [1.0, 0.984304, 0.015696, 0.0]])
    np.testing.assert_allclose(o.h, h1, rtol=1e-14, atol=1e-15)
    qx1 = np.zeros((4, 5))
    qx1[:, 2] = 0.15696
    qx1[1, 0] = -1.054092553389460
    np.testing.assert_allclose(o.qx, qx1, rtol=1e-14, atol=1e-15)
    assert np.all(o.qy == 0.0)
    o.run(1)
    h2 = np.array([[9.881195744512494e-1, 9.562893170728781e-1, 4.522629217791231e-2, 2.416834920960000e-5],
                   [8.363854586562135e-1, 9.460868075851215e-1, 4.522629217791231e-2, 2.416834920960000e-5],
                   [9.881195744512494e-1, 9.562893170728781e-1, 4.522629217791231e-2, 2.416834920960000e-5],
                   [9.984602224000000e-1, 9.562893170728781e-1, 4.522629217791231e-2, 2.416834920960000e-5]])
    np.testing.assert_allclose(o.h, h2, rtol=1e-13, atol=1e-16)
    qx2 = np.array([[0.0, 1.539777600000000e-2, 2.955446052712191e-1, 2.416834920960000e-4, 0.0],
                    [-8.754931379009831e-1, -8.662731887756611e-2, 2.955446052712191e-1, 2.416834920960000e-4, 0.0],
                    [0.0, 1.539777600000000e-2, 2.955446052712191e-1, 2.416834920960000e-4, 0.0],
                    [0.0, 1.539777600000000e-2, 2.955446052712191e-1, 2.416834920960000e-4, 0.0]])
    np.testing.assert_allclose(o.qx, qx2, rtol=1e-13, atol=1e-16)
    qy2 = np.zeros((5, 4))
    qy2[1, 0] = 1.034064794875060e-1
    qy2[2, 0] = -1.034064794875060e-1
    np.testing.assert_allclose(o.qy, qy2, rtol=1e-13, atol=1e-16)


# ---------------------------------------------------------------- P3: lake at rest
@pytest.mark.parametrize("shape", [(16, 16), (7, 5), (33, 17)])
def test_p3_lake_at_rest_is_exact(shape):
    """Flat water surface over dyadic terrain with dry islands stays bitwise at rest."""
    nx, ny = shape
    p = inputs.lake_at_rest(nx, ny)
    assert (p.z > 2.0).any() and (p.z < 2.0).any()   # both wet and dry cells
    o = oracle.Oracle(p)
    h0 = o.h.copy()
    o.run(200)
    assert np.array_equal(o.h, h0)
    assert not o.qx.any() and not o.qy.any()


def test_p3_lake_at_rest_fractal_cfl():
    p = inputs.c2_fractal(nx=64, ny=48, steps=10)
    z = p.z
    eta0 = float(np.quantile(z, 0.4))
    lake = Problem("lake_fractal", p.nx, p.ny, p.dx, z, p.n, [], Options(dt_cap=0.5),
                   h0=np.maximum(eta0 - z, 0.0))
    o = oracle.Oracle(lake)
    o.run(100)
    assert np.abs(o.qx).max() < 1e-12 and np.abs(o.qy).max() < 1e-12


# ---------------------------------------------------------------- linear standing waves
@pytest.mark.parametrize("nx,ny,mx,my,theta", [(16, 1, 3, 0, 1.0), (1, 12, 0, 2, 1.0), (12, 10, 2, 3, 1.0),
                                               (12, 10, 1, 2, 0.9), (16, 1, 3, 0, 0.8)])
def test_standing_waves_follow_the_discrete_dispersion_relation(nx, ny, mx, my, theta):
    """A standing wave of 1e-7 m on a 2 m lake (no friction, walls) against the
    closed form of the linearised scheme (closed_forms.standing_wave_amplitudes): x waves, y
    waves, an oblique mode, and the theta weighting.  Pins g, dt, dx and the
    signs of Eq. 3's slope term and of Eq. 4, the face/cell index pairing of
    both axes, and the theta factor.  The neglected terms are O(eps^2 / H) per
    step; measured at about 1e-7 eps over 120 steps, bound 1e-5 eps (a 0.1 %
    change of g alone moves the result by 8e-3 eps)."""
    H, eps, dx, dt, steps = 2.0, 1e-7, 1.5, 0.05, 120
    p = inputs.standing_wave(nx, ny, mx, my, H=H, eps=eps, dx=dx, dt=dt, theta=theta)
    mode = (p.h0 - H) / eps
    amp = standing_wave_amplitudes(nx, ny, mx, my, H, dx, dt, theta, steps)
    assert np.abs(amp).max() > 0.5           # the mode swings through several periods
    o = oracle.Oracle(p)
    for k in range(steps):
        o.run(1)
        assert np.abs((o.h - H) - eps * amp[k] * mode).max() < 1e-5 * eps, k


# ---------------------------------------------------------------- P4: mass ledger
def test_p4_mass_ledger_c1():
    """V(T) - V(0) = V_in - V_out + V_clip on the 128^2 channel run; V_in = sum dt Q."""
    p = inputs.c1_tilted_channel()
    o = oracle.Oracle(p)
    V0 = o.volume()
    _, dts = o.run(1000, dt_log=True)
    L = o.ledger_dict()
    assert L["V_in"] == pytest.approx(float(np.sum(dts * 50.0)), rel=1e-15)
    bal = o.volume() - V0 - (L["V_in"] - L["V_out"] + L["V_clip"])
    assert abs(bal) <= 1e-12 * L["V_in"]
    assert L["V_out"] > 0.0


def test_p4_mass_ledger_with_clipping():
    """Thin water at an outflow edge drains below zero; the clip volume closes the ledger."""
    z = np.zeros((6, 8))
    h0 = np.full((6, 8), 0.002)
    secs = [Section.cells(XMAX, 0, 6, OUTFLOW, 0.5, 8, 6), Section.cells(YMIN, 0, 8, OUTFLOW, 0.5, 8, 6)]
    o = oracle.Oracle(closed_box(z, h0, dx=0.1, n=0.01, sections=secs, dt_const=0.05))
    V0 = o.volume()
    o.run(20)
    L = o.ledger_dict()
    assert L["V_clip"] > 0.0
    assert np.all(o.h >= 0.0)
    bal = o.volume() - V0 - (L["V_in"] - L["V_out"] + L["V_clip"])
    assert abs(bal) <= 1e-12 * max(V0, L["V_out"])


@pytest.mark.parametrize("seed", [0, 1])
def test_p4_mass_ledger_random(seed):
    p = inputs.random_small(23, 17, seed)
    o = oracle.Oracle(p)
    V0 = o.volume()
    o.run(150)
    L = o.ledger_dict()
    assert L["V_in"] > 0 and L["V_out"] > 0
    bal = o.volume() - V0 - (L["V_in"] - L["V_out"] + L["V_clip"])
    assert abs(bal) <= 1e-12 * (V0 + L["V_in"])


# ---------------------------------------------------------------- P5: normal depth
def test_p5_uniform_channel_reaches_manning_normal_depth():
    """At steady state Eq. 3 reduces to q = h^(5/3) sqrt(S0) / n (Manning)."""
    p = inputs.normal_depth_channel(h_n=1.0)
    o = oracle.Oracle(p)
    for _ in range(60):
        prev = o.h.copy()
        o.run(500)
        if np.abs(o.h - prev).max() < 1e-13:
            break
    assert np.abs(o.h - 1.0).max() < 1e-6
    q_manning = math.sqrt(1e-3) / 0.03      # h_n = 1
    np.testing.assert_allclose(o.qx[:, 1:], q_manning, rtol=1e-9)
    assert np.abs(o.qy).max() < 1e-12


def test_p5_normal_depth_other_depth():
    h_n = 0.37
    p = inputs.normal_depth_channel(nx=40, ny=3, dx=5.0, S0=4e-3, n=0.05, h_n=h_n)
    p.h0 = np.full((3, 40), 0.5)
    o = oracle.Oracle(p)
    for _ in range(80):
        prev = o.h.copy()
        o.run(500)
        if np.abs(o.h - prev).max() < 1e-13:
            break
    assert np.abs(o.h - h_n).max() < 1e-6


# ---------------------------------------------------------------- P6: symmetry
def _mirror_y(p):
    ny = p.ny
    secs = []
    flip = {YMIN: YMAX, YMAX: YMIN, XMIN: XMIN, XMAX: XMAX}
    for s in p.sections:
        if s.side in (XMIN, XMAX):
            a, b = round(s.frac_start * ny), round(s.frac_end * ny)
            secs.append(Section.cells(s.side, ny - b, ny - a, s.kind, s.slope, p.nx, ny, s.t_s, s.q_m3s))
        else:
            secs.append(Section(flip[s.side], s.frac_start, s.frac_end, s.kind, s.slope, s.t_s, s.q_m3s))
    return Problem(p.name + "_my", p.nx, ny, p.dx, p.z[::-1].copy(), p.n[::-1].copy(), secs, p.opts,
                   h0=p.h0[::-1].copy(), qx0=p.qx0[::-1].copy(), qy0=-p.qy0[::-1].copy())


def _transpose(p):
    secs = []
    swap = {XMIN: YMIN, XMAX: YMAX, YMIN: XMIN, YMAX: XMAX}
    for s in p.sections:
        secs.append(Section(swap[s.side], s.frac_start, s.frac_end, s.kind, s.slope, s.t_s, s.q_m3s))
    return Problem(p.name + "_T", p.ny, p.nx, p.dx, p.z.T.copy(), p.n.T.copy(), secs, p.opts,
                   h0=p.h0.T.copy(), qx0=p.qy0.T.copy(), qy0=p.qx0.T.copy())


def _outflow_only(seed):
    p = inputs.random_small(19, 14, seed)
    p.sections = [s for s in p.sections if s.kind == OUTFLOW]
    return p


def test_p6_mirror_y_is_bitwise():
    """Reflecting y negates every y-face exactly and leaves Eq. 4's sums unchanged."""
    p = _outflow_only(3)
    a, b = oracle.Oracle(p), oracle.Oracle(_mirror_y(p))
    a.run(60)
    b.run(60)
    assert np.array_equal(a.h, b.h[::-1])
    assert np.array_equal(a.qx, b.qx[::-1])
    assert np.array_equal(a.qy, -b.qy[::-1])


def test_p6_transpose_with_inflow():
    """Swapping the axes swaps qx and qy; with inflow the Eq. 6 sums only reorder."""
    p = inputs.random_small(19, 14, 4)
    a, b = oracle.Oracle(p), oracle.Oracle(_transpose(p))
    a.run(60)
    b.run(60)
    np.testing.assert_allclose(a.h, b.h.T, rtol=0, atol=1e-12)
    np.testing.assert_allclose(a.qx, b.qy.T, rtol=0, atol=1e-12)
    np.testing.assert_allclose(a.qy, b.qx.T, rtol=0, atol=1e-12)


def test_p6_transpose_outflow_only_bitwise():
    p = _outflow_only(5)
    a, b = oracle.Oracle(p), oracle.Oracle(_transpose(p))
    a.run(40)
    b.run(40)
    assert np.array_equal(a.h, b.h.T)
    assert np.array_equal(a.qx, b.qy.T)


# ---------------------------------------------------------------- P8 and the dt rule
def test_p8_constant_dt_two_simulated_days():
    """0.1 s constant steps: 1.728 M steps make two simulated days (172 800 s)."""
    p = closed_box(np.zeros((1, 1)), [[0.0]], dt_const=0.1)
    o = oracle.Oracle(p)
    o.run(1_728_000)
    assert o.ledger.step == 1_728_000
    assert o.ledger.t == pytest.approx(172_800.0, rel=1e-9)


def test_cfl_rule_and_epochs():
    p = inputs.random_small(20, 12, 2)
    p.opts.epoch_steps = 5
    o = oracle.Oracle(p)
    hmax0 = o.h.max()
    _, dts = o.run(23, dt_log=True)
    # held constant inside each epoch of 5 steps
    for e in range(0, 23, 5):
        assert np.all(dts[e:e + 5] == dts[e])
    # Courant number alpha at the first epoch (unless capped)
    c = dts[0] * math.sqrt(9.81 * hmax0) / p.dx
    assert c == pytest.approx(0.7, rel=1e-14) or dts[0] == p.opts.dt_cap
    dry = oracle.Oracle(closed_box(np.zeros((3, 3)), np.zeros((3, 3)), dt_mode=0, dt_cap=1.5))
    assert dry.dt() == 1.5


# ---------------------------------------------------------------- final-step truncation
def _basin_with_inflow(t_s, q, **opt):
    """Closed flat 6 x 4 basin, 0.5 m of water, one inflow section on xmin (rows 1-2)."""
    sec = Section.cells(XMIN, 1, 3, INFLOW, 1e-3, 6, 4, t_s, q)
    return closed_box(np.zeros((4, 6)), np.full((4, 6), 0.5), sections=[sec], **opt)


def test_advance_lands_on_the_end_time_with_exact_inflow_volume():
    """Constant Q = 2 m^3/s, dt = 0.1 s: advancing 0.55 s takes ceil(5.5) = 6 steps,
    the last one 0.05 s long; the clock reads 0.55 exactly, V_in = Q x 0.55 and the
    stored volume grows by exactly V_in (closed basin, nothing leaves)."""
    o = oracle.Oracle(_basin_with_inflow([0.0, 100.0], [2.0, 2.0], dt_const=0.1))
    V0 = o.volume()
    assert o.advance(0.55) == 6
    assert o.ledger.t == 0.55
    assert o.ledger.V_in == pytest.approx(2.0 * 0.55, rel=1e-14)
    assert o.volume() - V0 == pytest.approx(o.ledger.V_in, rel=1e-12)
    assert o.ledger.V_out == 0.0 and o.ledger.V_clip == 0.0
    assert o.ledger.dt == 0.1                        # the epoch keeps its time step
    assert o.advance(0.55) == 0                      # already there
    with pytest.raises(ValueError):
        o.advance(0.5)


def test_advance_truncated_step_uses_its_start_time_and_length():
    """Q(t) = 10 t, dt = 1 s, advance to 2.5 s: steps start at 0, 1, 2 with lengths
    1, 1, 0.5, so V_in = Q(0)*1 + Q(1)*1 + Q(2)*0.5 = 20 m^3 (a full last step would
    give 30, a last step sampled at its end 22.5)."""
    o = oracle.Oracle(_basin_with_inflow([0.0, 100.0], [0.0, 1000.0], dt_const=1.0))
    assert o.advance(2.5) == 3
    assert o.ledger.V_in == pytest.approx(20.0, rel=1e-14)


def test_advance_in_cfl_epochs_keeps_the_books():
    """CFL epochs of 4 steps: several advances to arbitrary times land on them
    exactly, with constant inflow into the closed basin V_in = Q (t - t0), and the
    ledger closes (V - V0 = V_in + V_clip, nothing leaves)."""
    o = oracle.Oracle(_basin_with_inflow([0.0, 1e4], [3.0, 3.0], dt_mode=0, dt_cap=0.7, epoch_steps=4))
    V0 = o.volume()
    for T in (0.3, 1.9, 2.0, 7.777):
        o.advance(T)
        assert o.ledger.t == T
    assert o.ledger.V_in == pytest.approx(3.0 * 7.777, rel=1e-13)
    assert o.ledger.V_out == 0.0
    assert o.volume() - V0 == pytest.approx(o.ledger.V_in + o.ledger.V_clip, rel=1e-12)


# ---------------------------------------------------------------- theta-weighted faces
def test_theta_scheme_hand_values_one_row():
    """de Almeida's theta weighting, theta = 0.7, one step on a row of 4 cells:
    flat bed, h = (1.0, 0.9, 0.8, 0.7), faces (0, 0.2, 0.1, 0.05, 0) with closed
    ends, n = 0.03, dt = 0.1 s, dx = 1 m.  Numerator discharge of face i:
    0.7 q_i + 0.15 (q_{i-1} + q_{i+1}); friction with |q_i| itself.  Literals:
    40-digit decimal evaluation of those formulas, done by hand."""
    p = closed_box(np.zeros((1, 4)), [[1.0, 0.9, 0.8, 0.7]], theta=0.7, n=0.03)
    p.qx0 = np.array([[0.0, 0.2, 0.1, 0.05, 0.0]])
    o = oracle.Oracle(p)
    o.run(1)
    np.testing.assert_allclose(o.qx[0, 1:4], [0.2530553154923903537113417, 0.1957678985649310959148924,
                                              0.1284704542920134320134527], rtol=1e-14)
    np.testing.assert_allclose(o.h[0], [0.9746944684507609646288658, 0.9057287416927459257796449,
                                        0.8067297444272917663901440, 0.7128470454292013432013453], rtol=1e-14)


@pytest.mark.parametrize("theta", [1.0, 0.9, 0.7, 0.55])
def test_theta_scheme_uniform_and_checkerboard_fluxes(theta):
    """Flat water surface, no friction: the slope term vanishes and a face keeps
    theta q + (1 - theta)/2 (q_prev + q_next).  A uniform flux field (faces away
    from the walls) is kept exactly; a field alternating +a, -a from face to face
    is scaled by 2 theta - 1 per step (the damping of the theta scheme)."""
    nx = 12
    z = np.zeros((1, nx))
    h0 = np.full((1, nx), 2.0)
    uni = closed_box(z, h0, theta=theta, n=0.0)
    uni.qx0 = np.concatenate([[0.0], np.full(nx - 1, 0.3), [0.0]])[None, :]
    o = oracle.Oracle(uni)
    o.step_dt(1e-9)                     # a step too short to change the depths measurably
    np.testing.assert_allclose(o.qx[0, 2:nx - 1], 0.3, rtol=1e-14)
    chk = closed_box(z, h0, theta=theta, n=0.0)
    a = 0.2 * (-1.0) ** np.arange(nx + 1)
    a[0] = a[-1] = 0.0
    chk.qx0 = a[None, :]
    o = oracle.Oracle(chk)
    o.step_dt(1e-9)
    np.testing.assert_allclose(o.qx[0, 2:nx - 1], (2 * theta - 1) * a[2:nx - 1], rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("friction", [0, 1])
def test_friction_norm_closed_form(friction):
    """Flat water 1 m deep, n = 0.05, dt = 0.1 s, every old x-face carries 0.3 and
    every y-face 0.4 m^2/s.  No slope term, so a face keeps q / (1 + g dt n^2 |q|):
    |q| is the face's own component (0.3 or 0.4) by default, and the vector norm
    sqrt(0.3^2 + 0.4^2) = 0.5 with the orthogonal mean of the four faces around it."""
    nx, ny = 5, 4
    p = closed_box(np.zeros((ny, nx)), np.ones((ny, nx)), n=0.05, friction=friction)
    p.qx0 = np.full((ny, nx + 1), 0.3)
    p.qy0 = np.full((ny + 1, nx), 0.4)
    o = oracle.Oracle(p)
    o.step_dt(0.1)
    c = 9.81 * 0.1 * 0.05 ** 2
    mx, my = (0.5, 0.5) if friction else (0.3, 0.4)
    np.testing.assert_allclose(o.qx[:, 1:nx], 0.3 / (1 + c * mx), rtol=1e-14)
    np.testing.assert_allclose(o.qy[1:ny, :], 0.4 / (1 + c * my), rtol=1e-14)


def test_friction_vector_norm_takes_the_four_faces_around():
    """Flat water 1 m deep (h_f = 1, no slope term), n = 0.05, dt = 0.1 s.  Old
    x-face discharges 0.3 + 0.1 j (rising with the row), y-face discharges
    0.4 + 0.2 i (rising with the column).  The four y-faces around x-face (j, i)
    (between cells i - 1 and i) sit in columns i - 1 and i, mean
    0.4 + 0.2 (i - 1/2); the four x-faces around y-face (j, i) sit in rows j - 1
    and j, mean 0.3 + 0.1 (j - 1/2).  A face keeps q / (1 + g dt n^2 sqrt(q^2 + mean^2));
    a mean taken one column or row off moves it by about 1e-4 of q."""
    nx, ny = 6, 5
    p = closed_box(np.zeros((ny, nx)), np.ones((ny, nx)), n=0.05, friction=1)
    jj, ii = np.mgrid[0:ny, 0:nx + 1]
    p.qx0 = 0.3 + 0.1 * jj
    jj, ii = np.mgrid[0:ny + 1, 0:nx]
    p.qy0 = 0.4 + 0.2 * ii
    o = oracle.Oracle(p)
    o.step_dt(0.1)
    c = 9.81 * 0.1 * 0.05 ** 2
    for j in range(ny):
        for i in range(1, nx):
            q, m = 0.3 + 0.1 * j, 0.4 + 0.2 * (i - 0.5)
            assert o.qx[j, i] == pytest.approx(q / (1 + c * math.sqrt(q * q + m * m)), rel=1e-14), (j, i)
    for j in range(1, ny):
        for i in range(nx):
            q, m = 0.4 + 0.2 * i, 0.3 + 0.1 * (j - 0.5)
            assert o.qy[j, i] == pytest.approx(q / (1 + c * math.sqrt(q * q + m * m)), rel=1e-14), (j, i)


# ---------------------------------------------------------------- boundary conditions
def test_section_fraction_rule():
    p = inputs.random_small(20, 12, 0)
    o = oracle.Oracle(p)
    ny, nx = 12, 20
    assert o.section_range(0) == (ny // 4, 3 * ny // 4)
    assert o.section_range(1) == (nx // 3, 2 * nx // 3)
    assert o.section_range(2) == (0, ny)


def test_hydrograph_matches_numpy_interp():
    p = inputs.random_small(10, 10, 0)
    o = oracle.Oracle(p)
    s = p.sections[0]
    for t in [-5.0, 0.0, 12.5, 50.0, 77.7, 200.0, 1e6]:
        assert o.hydrograph(0, t) == pytest.approx(np.interp(t, s.t_s, s.q_m3s), rel=1e-15, abs=1e-15)


@pytest.mark.parametrize("bc_form", [0, 1])
def test_inflow_uniform_section_splits_evenly(bc_form):
    """Equal bed levels and roughness: every section cell carries Q / (m dx)."""
    z = np.full((9, 5), 3.0)
    secs = [Section.cells(XMIN, 2, 7, INFLOW, 1e-3, 5, 9, [0, 1], [12.0, 12.0])]
    o = oracle.Oracle(closed_box(z, np.zeros((9, 5)), dx=2.0, sections=secs, bc_form=bc_form))
    W, q = o.inflow_faces(0, 12.0)
    np.testing.assert_allclose(q, 12.0 / (5 * 2.0), rtol=1e-14)
    # Eq. 5 at that level gives the same per-cell discharge (closed form)
    hh = W - 3.0
    per_cell = (2.0 * hh ** (5 / 3) if bc_form == 0 else 4.0 * hh ** (2 / 3)) * math.sqrt(1e-3) / 0.03
    assert per_cell == pytest.approx(12.0 / 5, rel=1e-9)


@pytest.mark.parametrize("bc_form", [0, 1])
def test_inflow_level_matches_brentq(bc_form):
    """W solves sum_c Q_c(W) = Q_in (Eq. 6); check against scipy's root finder."""
    from scipy.optimize import brentq
    rng = np.random.default_rng(11)
    z = rng.uniform(0.0, 2.0, (10, 6))
    n = rng.uniform(0.02, 0.08, (10, 6))
    p = closed_box(z, np.zeros((10, 6)), dx=3.0, sections=[
        Section.cells(YMAX, 1, 5, INFLOW, 2e-3, 6, 10, [0, 1], [7.0, 7.0])], bc_form=bc_form)
    p.n = n
    o = oracle.Oracle(p)
    W, q = o.inflow_faces(0, 7.0)
    zc, nc = z[-1, 1:5], n[-1, 1:5]
    pe = 5 / 3 if bc_form == 0 else 2 / 3
    A = 3.0 if bc_form == 0 else 9.0

    def F(w):
        return np.sum(A * np.maximum(w - zc, 0.0) ** pe * math.sqrt(2e-3) / nc) - 7.0
    Wref = brentq(F, zc.min(), zc.min() + 100.0, xtol=1e-14, rtol=1e-15)
    assert W == pytest.approx(Wref, abs=2e-12)
    assert np.sum(q) * 3.0 == pytest.approx(7.0, rel=1e-14)
    assert np.all(q[zc >= W] == 0.0)


def test_outflow_literal_form_hand_value():
    """bc_form 1 (A = dx^2 in Eq. 5): unit-width flux dx h^(2/3) sqrt(S)/n."""
    z = np.zeros((1, 1))
    secs = [Section.cells(XMAX, 0, 1, OUTFLOW, 4e-4, 1, 1)]
    o = oracle.Oracle(closed_box(z, [[0.512]], dx=2.0, n=0.04, sections=secs, bc_form=1, dt_const=0.01))
    o.run(1)
    # 2 * 0.512^(2/3) * 0.02 / 0.04 = 2 * 0.64 * 0.5 = 0.64 m^2/s
    assert o.qx[0, 1] == pytest.approx(0.64, rel=1e-14)
    assert o.h[0, 0] == pytest.approx(0.512 - 0.01 * 0.64 / 2.0, rel=1e-14)


# ---------------------------------------------------------------- adjoint
def wet_case(nx=12, ny=9, seed=0, bc_form=0, theta=1.0, friction=0):
    rng = np.random.default_rng(500 + seed)
    dx = 4.0
    xm = (np.arange(nx) + 0.5) * dx
    z = 1.0 - 2e-3 * xm[None, :] + rng.uniform(-0.05, 0.05, (ny, nx))
    h0 = 0.6 + rng.uniform(0.0, 0.2, (ny, nx))
    n = rng.uniform(0.03, 0.06, (ny, nx))
    so = 2e-3 if bc_form == 0 else 2e-5      # the literal form drains ~dx/h times faster
    secs = [Section.cells(XMIN, 2, 7, INFLOW, 2e-3, nx, ny, [0.0, 30.0], [1.0, 3.0]),
            Section.cells(XMAX, 0, ny, OUTFLOW, so, nx, ny),
            Section.cells(YMAX, 3, 8, OUTFLOW, so / 2, nx, ny)]
    p = Problem("wet", nx, ny, dx, z, n, secs,
                Options(dt_mode=1, dt_const=0.4, bc_form=bc_form, theta=theta, friction=friction), h0=h0,
                qx0=np.zeros((ny, nx + 1)), qy0=np.zeros((ny + 1, nx)))
    return p


def _loss(p, n, steps, gauges, w):
    p2 = Problem(p.name, p.nx, p.ny, p.dx, p.z, n, p.sections, p.opts, h0=p.h0, qx0=p.qx0, qy0=p.qy0)
    o = oracle.Oracle(p2)
    series, _ = o.run(steps, gauges=gauges)
    assert o.h.min() > 0.05
    return float(np.sum(series * w))


@pytest.mark.parametrize("bc_form,theta,friction", [(0, 1.0, 0), (1, 1.0, 0), (0, 0.8, 0), (0, 1.0, 1),
                                                     (0, 0.8, 1), (1, 0.85, 1)])
def test_adjoint_dn_matches_central_differences(bc_form, theta, friction):
    """dL/dn by the reverse sweep equals central finite differences of the forward run,
    for Eq. 3 as printed and its theta-weighted and vector-norm forms."""
    p = wet_case(bc_form=bc_form, theta=theta, friction=friction)
    steps = 40
    rng = np.random.default_rng(3)
    gauges = np.array([[3, 4], [8, 2], [10, 7], [0, 4], [11, 0]])
    w = rng.standard_normal((steps, len(gauges)))
    o = oracle.Oracle(p)
    gn = o.adjoint(steps, gauges, w)
    cells = [(0, 3), (0, 5), (4, 4), (11, 2), (6, 8), (3, 0), (7, 6), (11, 8)]  # incl. inflow + outflow cells
    for (i, j) in cells:
        eps = 1e-4 * p.n[j, i]      # the W bisection's 1e-12 m bracket is FD noise below ~1e-5
        npl, nmi = p.n.copy(), p.n.copy()
        npl[j, i] += eps
        nmi[j, i] -= eps
        fd = (_loss(p, npl, steps, gauges, w) - _loss(p, nmi, steps, gauges, w)) / (2 * eps)
        assert gn[j, i] == pytest.approx(fd, rel=1e-5, abs=1e-9 * np.abs(gn).max())


@pytest.mark.parametrize("theta,friction", [(1.0, 0), (0.8, 0), (1.0, 1), (0.8, 1)])
def test_adjoint_dh0_matches_central_differences(theta, friction):
    """dL/d(h0, qx0, qy0) against central differences; with the vector norm the
    faces of one axis also reach the other axis's faces, and with the theta
    weighting a face's neighbours along its axis (the boundary faces included)."""
    p = wet_case(seed=1, theta=theta, friction=friction)
    rng = np.random.default_rng(11)
    p.qx0 = rng.uniform(-0.05, 0.05, (p.ny, p.nx + 1))     # moving water: |q| and the vector norm are smooth
    p.qy0 = rng.uniform(-0.05, 0.05, (p.ny + 1, p.nx))
    p.qx0[:, 0] = 0.0
    p.qy0[-1, :] = 0.0
    steps = 30
    gauges = np.array([[5, 5], [9, 3]])
    w = np.ones((steps, 2))
    o = oracle.Oracle(p)
    gn, lh, lqx, lqy = o.adjoint(steps, gauges, w, want_state=True)

    def fd(field, j, i, eps=1e-6):
        vals = []
        for sgn in (1, -1):
            p2 = wet_case(seed=1, theta=theta, friction=friction)
            p2.h0, p2.qx0, p2.qy0 = p.h0.copy(), p.qx0.copy(), p.qy0.copy()
            getattr(p2, field)[j, i] += sgn * eps
            s, _ = oracle.Oracle(p2).run(steps, gauges=gauges)
            vals.append(np.sum(s * w))
        return (vals[0] - vals[1]) / (2 * eps)

    for (i, j) in [(5, 5), (2, 2), (10, 6), (0, 0)]:
        assert lh[j, i] == pytest.approx(fd("h0", j, i), rel=2e-5, abs=1e-8)
    for (j, i) in [(4, 6), (5, 1), (3, 0)]:           # interior x-faces, and a boundary face's old value
        assert lqx[j, i] == pytest.approx(fd("qx0", j, i), rel=2e-5, abs=1e-8)
    for (j, i) in [(4, 6), (2, 9)]:                    # interior y-faces
        assert lqy[j, i] == pytest.approx(fd("qy0", j, i), rel=2e-5, abs=1e-8)


def _dot_case(theta, friction, bc_form, inflow):
    """10 x 7 wet basin with moving water (|q| and the vector norm smooth),
    outflow on three sides and optionally a Manning inflow section."""
    rng = np.random.default_rng(900)
    nx, ny, dx = 10, 7, 4.0
    xm = (np.arange(nx) + 0.5) * dx
    z = 1.0 - 2e-3 * xm[None, :] + rng.uniform(-0.05, 0.05, (ny, nx))
    h0 = 0.6 + rng.uniform(0.0, 0.2, (ny, nx))
    n = rng.uniform(0.03, 0.06, (ny, nx))
    so = 2e-3 if bc_form == 0 else 2e-5
    secs = [Section.cells(XMAX, 0, ny, OUTFLOW, so, nx, ny), Section.cells(YMAX, 3, 8, OUTFLOW, so / 2, nx, ny),
            Section.cells(YMIN, 0, 4, OUTFLOW, so, nx, ny)]
    if inflow:
        secs.append(Section.cells(XMIN, 2, 6, INFLOW, 2e-3, nx, ny, [0.0, 30.0], [1.0, 3.0]))
    return Problem("dot", nx, ny, dx, z, n, secs,
                   Options(dt_mode=1, dt_const=0.4, bc_form=bc_form, theta=theta, friction=friction), h0=h0,
                   qx0=rng.uniform(-0.05, 0.05, (ny, nx + 1)), qy0=rng.uniform(-0.05, 0.05, (ny + 1, nx)))


@pytest.mark.parametrize("theta,friction,bc_form,inflow", [(1.0, 0, 0, False), (0.8, 0, 0, False),
                                                           (1.0, 1, 0, False), (0.85, 1, 1, False),
                                                           (1.0, 0, 0, True)])
def test_adjoint_dot_product_one_step(theta, friction, bc_form, inflow):
    """The transpose test on one step y = S(x), x = (h, qx, qy, n): for a random
    seed lam on the depths after the step and a random direction v,
    <lam, J v> = <J^T lam, v>.  J^T lam is the reverse sweep's (dL/dh0, dL/dqx0,
    dL/dqy0, dL/dn) with L = <lam, h(after the step)>; J v is the fourth-order
    central difference of L along v (step 5e-3 of v: truncation and rounding
    both near 1e-12 of the product, masks fixed on this range).  Agreement to
    1e-10 relative, for each input separately, checks every term of the
    reverse step far below the per-cell finite differences' 1e-5."""
    p = _dot_case(theta, friction, bc_form, inflow)
    rng = np.random.default_rng(5)
    lam = rng.standard_normal((p.ny, p.nx))
    jj, ii = np.mgrid[0:p.ny, 0:p.nx]
    gauges = np.stack([ii.ravel(), jj.ravel()], 1)
    gn, lh, lqx, lqy = oracle.Oracle(p).adjoint(1, gauges, lam.reshape(1, -1), want_state=True)
    full = (0.01 * rng.standard_normal(p.h0.shape), 0.01 * rng.standard_normal(p.qx0.shape),
            0.01 * rng.standard_normal(p.qy0.shape), 0.001 * rng.standard_normal(p.n.shape))
    grads = (lh, lqx, lqy, gn)

    def L(v, e):
        q = Problem(p.name, p.nx, p.ny, p.dx, p.z, p.n + e * v[3], p.sections, p.opts, h0=p.h0 + e * v[0],
                    qx0=p.qx0 + e * v[1], qy0=p.qy0 + e * v[2])
        o = oracle.Oracle(q)
        o.run(1)
        return float(np.sum(lam * o.h))
    e = 5e-3
    for k in range(4):                  # one input at a time (h, qx, qy, n), each to its own 1e-10
        v = tuple(full[m] if m == k else np.zeros_like(full[m]) for m in range(4))
        transposed = float(np.sum(grads[k] * v[k]))
        tangent = (8.0 * (L(v, e) - L(v, -e)) - (L(v, 2 * e) - L(v, -2 * e))) / (12.0 * e)
        assert abs(transposed) > 1e-6, k
        assert transposed == pytest.approx(tangent, rel=1e-10), k


@pytest.mark.parametrize("nx,ny,mx,my,theta", [(16, 1, 3, 0, 1.0), (12, 10, 2, 3, 1.0), (12, 10, 1, 2, 0.9),
                                               (1, 12, 0, 2, 0.8), (16, 1, 3, 0, 0.7)])
def test_adjoint_at_rest_is_the_transposed_mode_dynamics(nx, ny, mx, my, theta):
    """A 2 m lake at rest (n = 0.03, walls): there the reverse sweep's Jacobian is
    the linear staggered scheme's (no discharge, so neither friction nor the
    h_f factor of the slope term has a derivative), and the gradient of
    L = <cosine mode, depths after 40 steps> has the closed form of
    closed_forms.standing_wave_gradient: the mode dynamics transposed, plus the
    wall faces' theta terms.  dL/dn is zero.  Bound 1e-12 (measured 1e-15)."""
    H, dx, dt, steps = 2.0, 1.5, 0.05, 40
    p = inputs.standing_wave(nx, ny, mx, my, H=H, eps=0.0, dx=dx, dt=dt, theta=theta, n=0.03)
    mh, gh, gx, gy = standing_wave_gradient(nx, ny, mx, my, H, dx, dt, theta, steps)
    jj, ii = np.mgrid[0:ny, 0:nx]
    gauges = np.stack([ii.ravel(), jj.ravel()], 1)
    seed = np.zeros((steps, nx * ny))
    seed[-1] = mh.ravel()
    gn, lh, lqx, lqy = oracle.Oracle(p).adjoint(steps, gauges, seed, want_state=True)
    assert np.abs(gh).max() > 0.1
    np.testing.assert_allclose(lh, gh, rtol=0, atol=1e-12)
    np.testing.assert_allclose(lqx, gx, rtol=0, atol=1e-12)
    np.testing.assert_allclose(lqy, gy, rtol=0, atol=1e-12)
    assert not gn.any()


def test_adjoint_zero_seed_gives_zero():
    p = wet_case()
    o = oracle.Oracle(p)
    gn = o.adjoint(10, np.array([[1, 1]]), np.zeros((10, 1)))
    assert not gn.any()
