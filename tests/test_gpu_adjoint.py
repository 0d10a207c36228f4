"""GPU adjoint (flood_adjoint) against the FP64 oracle's reverse sweep, finite
differences and its own store-all run.

Tolerances: FP64 GPU vs FP64 oracle 1e-9 of max|dL/dn| (same arithmetic up
to cbrt ulps and summation order); revolve vs store-all bitwise (the replays
are deterministic); FP32 GPU vs FP64 oracle 1e-2 relative with cosine
similarity > 0.999; FD checks 1e-5 relative in FP64, 1e-2 for the FP32
adjoint at full size.
"""
import math

import numpy as np
import pytest

import inputs
from inputs import INFLOW, OUTFLOW, XMAX, XMIN, YMAX, YMIN, Options, Problem, Section
import oracle

pytestmark = pytest.mark.gpu


def F():
    import paper_2204_10323_gb300 as F
    return F


def wet_case(nx=24, ny=17, seed=0, bc_form=0, dt_mode=1, E=4, theta=1.0, friction=0, moving=False):
    rng = np.random.default_rng(700 + seed)
    dx = 4.0
    xm = (np.arange(nx) + 0.5) * dx
    z = 1.0 - 2e-3 * xm[None, :] + rng.uniform(-0.05, 0.05, (ny, nx))
    h0 = 0.6 + rng.uniform(0.0, 0.2, (ny, nx))
    n = rng.uniform(0.03, 0.06, (ny, nx))
    so = 2e-3 if bc_form == 0 else 2e-5
    secs = [Section.cells(XMIN, 2, ny - 3, INFLOW, 2e-3, nx, ny, [0.0, 30.0], [1.0, 3.0]),
            Section.cells(XMAX, 0, ny, OUTFLOW, so, nx, ny),
            Section.cells(YMAX, 3, nx - 4, OUTFLOW, so / 2, nx, ny)]
    qx0, qy0 = np.zeros((ny, nx + 1)), np.zeros((ny + 1, nx))
    if moving:                                   # moving water: |q| and the vector norm away from 0
        qx0 = rng.uniform(-0.05, 0.05, (ny, nx + 1))
        qy0 = rng.uniform(-0.05, 0.05, (ny + 1, nx))
        qx0[:, 0] = qy0[-1, :] = 0.0
    return Problem("wet", nx, ny, dx, z, n, secs,
                   Options(dt_mode=dt_mode, dt_const=0.4, dt_cap=0.4, epoch_steps=E, bc_form=bc_form,
                           theta=theta, friction=friction),
                   h0=h0, qx0=qx0, qy0=qy0)


def closed_cost(l, c):
    if l <= 1:
        return 0
    r = 0
    while math.comb(c + r, c) < l:
        r += 1
    return r * l - math.comb(c + r, c + 1)


GAUGES = np.array([[3, 4], [20, 2], [10, 11], [0, 8], [23, 0], [12, 16]])


@pytest.mark.parametrize("bc_form,dt_mode", [(0, 1), (1, 1), (0, 0)])
def test_fp64_adjoint_matches_oracle(bc_form, dt_mode):
    Fm = F()
    p = wet_case(bc_form=bc_form, dt_mode=dt_mode)
    steps = 37
    w = np.random.default_rng(5).standard_normal((steps, len(GAUGES)))
    o = oracle.Oracle(p)
    gn_o, lh_o, _, _ = o.adjoint(steps, GAUGES, w, want_state=True)
    s = Fm.Sim(p, precision=Fm.F64)
    gn, lh = s.adjoint(steps, GAUGES, w, n_checkpoints=steps, want_dh0=True)
    scale = np.abs(gn_o).max()
    assert scale > 0
    assert np.abs(gn - gn_o).max() <= 1e-9 * scale
    assert np.abs(lh - lh_o).max() <= 1e-9 * np.abs(lh_o).max()


@pytest.mark.parametrize("theta,friction,bc_form,dt_mode", [(0.8, 0, 0, 1), (1.0, 1, 0, 1), (0.8, 1, 0, 0),
                                                             (0.9, 1, 1, 1)])
def test_fp64_option_adjoint_matches_oracle(theta, friction, bc_form, dt_mode):
    """The theta-weighted and vector-norm forms: dL/dn and dL/d(h0, qx0, qy0) of the
    three-pass reverse step against the oracle's reverse sweep."""
    Fm = F()
    p = wet_case(bc_form=bc_form, dt_mode=dt_mode, theta=theta, friction=friction, moving=True, seed=8)
    steps = 33
    w = np.random.default_rng(9).standard_normal((steps, len(GAUGES)))
    o = oracle.Oracle(p)
    gn_o, lh_o, _, _ = o.adjoint(steps, GAUGES, w, want_state=True)
    s = Fm.Sim(p, precision=Fm.F64)
    gn, lh = s.adjoint(steps, GAUGES, w, n_checkpoints=5, want_dh0=True)
    assert np.abs(gn - gn_o).max() <= 1e-9 * np.abs(gn_o).max()
    assert np.abs(lh - lh_o).max() <= 1e-9 * np.abs(lh_o).max()
    # revolve and store-all give the same bits
    ref = s.adjoint(steps, GAUGES, w, n_checkpoints=steps)
    assert np.array_equal(ref, gn)


@pytest.mark.parametrize("theta,friction", [(0.8, 0), (1.0, 1), (0.8, 1)])
def test_fp32_option_adjoint_is_close_to_fp64(theta, friction):
    Fm = F()
    p = wet_case(theta=theta, friction=friction, moving=True, seed=10, nx=70, ny=45)
    steps = 40
    w = np.random.default_rng(11).standard_normal((steps, len(GAUGES)))
    g64 = Fm.Sim(p, precision=Fm.F64).adjoint(steps, GAUGES, w, n_checkpoints=6)
    q = Problem(p.name, p.nx, p.ny, p.dx, p.z.astype(np.float32).astype(np.float64),
                p.n.astype(np.float32).astype(np.float64), p.sections, p.opts,
                h0=p.h0.astype(np.float32).astype(np.float64), qx0=p.qx0.astype(np.float32).astype(np.float64),
                qy0=p.qy0.astype(np.float32).astype(np.float64))
    g32 = Fm.Sim(q, precision=Fm.F32).adjoint(steps, GAUGES, w, n_checkpoints=6).astype(np.float64)
    cos = float(np.sum(g32 * g64) / (np.linalg.norm(g32) * np.linalg.norm(g64)))
    assert cos > 0.999
    assert np.abs(g32 - g64).max() <= 1e-2 * np.abs(g64).max()


def test_fp64_adjoint_from_mid_epoch_state():
    """Start the reverse sweep from a state reached mid-epoch (CFL epochs of 4)."""
    Fm = F()
    p = wet_case(dt_mode=0, E=4, seed=2)
    o = oracle.Oracle(p)
    o.run(3)
    s = Fm.Sim(p, precision=Fm.F64)
    s.step(3)
    steps = 21
    w = np.random.default_rng(6).standard_normal((steps, len(GAUGES)))
    gn_o = o.adjoint(steps, GAUGES, w)
    gn = s.adjoint(steps, GAUGES, w, n_checkpoints=5)
    assert np.abs(gn - gn_o).max() <= 1e-9 * np.abs(gn_o).max()


@pytest.mark.parametrize("checkpoints", [1, 2, 3, 7])
def test_revolve_equals_store_all_and_costs_the_binomial_minimum(checkpoints):
    Fm = F()
    p = wet_case(seed=3)
    steps = 45
    w = np.random.default_rng(7).standard_normal((steps, len(GAUGES)))
    s = Fm.Sim(p, precision=Fm.F64)
    ref = s.adjoint(steps, GAUGES, w, n_checkpoints=steps)
    assert s.adjoint_forward_steps() == steps - 1
    gn = s.adjoint(steps, GAUGES, w, n_checkpoints=checkpoints)
    assert np.array_equal(gn, ref)
    assert s.adjoint_forward_steps() == closed_cost(steps, checkpoints)


@pytest.mark.parametrize("prec", ["F32", "F64"])
def test_automatic_checkpoints_keep_every_state(prec):
    # n_checkpoints = 0 sizes the snapshots by the free device memory: this small
    # grid keeps all of them, so it replays like store-all and gives its bits
    Fm = F()
    p = wet_case(seed=3)
    steps = 45
    w = np.random.default_rng(9).standard_normal((steps, len(GAUGES)))
    s = Fm.Sim(p, precision=getattr(Fm, prec))
    ref = s.adjoint(steps, GAUGES, w, n_checkpoints=steps)
    gn = s.adjoint(steps, GAUGES, w, n_checkpoints=0)
    assert s.adjoint_forward_steps() == steps - 1
    assert np.array_equal(gn, ref)
    assert np.array_equal(s.adjoint(steps, GAUGES, w, n_checkpoints=3), ref)


def test_automatic_checkpoints_halve_when_the_snapshot_block_fails():
    # n_checkpoints = 0 asks for one snapshot per step (45 here); the sweep's first
    # allocation, the snapshot block, is made to fail once, so the count halves to
    # 22 and the sweep goes on with the binomial schedule of 22 snapshots
    Fm = F()
    p = wet_case(seed=3)
    steps = 45
    w = np.random.default_rng(9).standard_normal((steps, len(GAUGES)))
    s = Fm.Sim(p, precision=Fm.F32)
    ref = s.adjoint(steps, GAUGES, w, n_checkpoints=steps)
    Fm.flood_debug_fail_alloc_after(0)
    try:
        gn = s.adjoint(steps, GAUGES, w, n_checkpoints=0)
    finally:
        Fm.flood_debug_fail_alloc_after(-1)
    assert s.adjoint_forward_steps() == closed_cost(steps, steps // 2)
    assert np.array_equal(gn, ref)
    s.close()


def test_adjoint_leaves_the_handle_unchanged():
    Fm = F()
    p = wet_case(seed=4, dt_mode=0)
    s = Fm.Sim(p)
    s.step(6)
    before = [a.copy() for a in s.state()]
    L0 = s.ledger()
    s.adjoint(30, GAUGES, np.ones((30, len(GAUGES))), n_checkpoints=4)
    after = s.state()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    L1 = s.ledger()
    for k in ("t", "dt", "V_in", "V_out", "V_clip", "step"):
        assert L1[k] == L0[k]
    # and stepping continues exactly as without the adjoint call
    t = Fm.Sim(p)
    t.step(6)
    s.step(11)
    t.step(11)
    assert np.array_equal(s.read(Fm.FIELD_H), t.read(Fm.FIELD_H))


def test_fp32_adjoint_close_to_fp64_oracle():
    Fm = F()
    p = wet_case(seed=5)
    p32 = Problem(p.name, p.nx, p.ny, p.dx, p.z.astype(np.float32).astype(np.float64),
                  p.n.astype(np.float32).astype(np.float64), p.sections, p.opts,
                  h0=p.h0.astype(np.float32).astype(np.float64), qx0=p.qx0, qy0=p.qy0)
    steps = 40
    w = np.random.default_rng(8).standard_normal((steps, len(GAUGES)))
    gn_o = oracle.Oracle(p32).adjoint(steps, GAUGES, w)
    gn = Fm.Sim(p32, precision=Fm.F32).adjoint(steps, GAUGES, w, n_checkpoints=6).astype(np.float64)
    cos = float(np.sum(gn * gn_o) / (np.linalg.norm(gn) * np.linalg.norm(gn_o)))
    assert cos > 0.999
    big = np.abs(gn_o) > 1e-2 * np.abs(gn_o).max()
    rel = np.abs(gn[big] - gn_o[big]) / np.abs(gn_o[big])
    assert np.median(rel) < 1e-3 and rel.max() < 1e-2


def test_fp32_adjoint_two_inflow_sections_sharing_a_corner():
    # two inflow sections meeting at cell (0, 0) (its west and its south face) on a
    # grid of 3 x 6 reverse-step tiles: the FP32 step's inflow blocks, one per section,
    # run beside the tiles, and their per-cell terms (the corner cell twice) join dL/dn
    # after the sweep; against the FP64 oracle's reverse sweep
    Fm = F()
    base = wet_case(nx=70, ny=45, seed=11)
    nx, ny = base.nx, base.ny
    secs = [Section.cells(XMIN, 0, 9, INFLOW, 2e-3, nx, ny, [0.0, 30.0], [1.0, 3.0]),
            Section.cells(YMIN, 0, 12, INFLOW, 2e-3, nx, ny, [0.0, 30.0], [2.0, 0.5]),
            Section.cells(XMAX, 0, ny, OUTFLOW, 2e-3, nx, ny)]
    r32 = lambda a: a.astype(np.float32).astype(np.float64)
    p = Problem("two_inflows", nx, ny, base.dx, r32(base.z), r32(base.n), secs, base.opts, h0=r32(base.h0),
                qx0=base.qx0, qy0=base.qy0)
    gauges = np.array([[1, 1], [0, 5], [6, 0], [30, 20], [69, 44], [3, 2]])
    steps = 32
    w = np.random.default_rng(12).standard_normal((steps, len(gauges)))
    gn_o = oracle.Oracle(p).adjoint(steps, gauges, w)
    gn = Fm.Sim(p, precision=Fm.F32).adjoint(steps, gauges, w, n_checkpoints=5).astype(np.float64)
    cos = float(np.sum(gn * gn_o) / (np.linalg.norm(gn) * np.linalg.norm(gn_o)))
    assert cos > 0.999
    sec = np.zeros((ny, nx), bool)
    sec[:9, 0] = True
    sec[0, :12] = True
    big = sec & (np.abs(gn_o) > 1e-3 * np.abs(gn_o).max())
    assert big.sum() >= 10
    rel = np.abs(gn[big] - gn_o[big]) / np.abs(gn_o[big])
    assert np.median(rel) < 1e-3 and rel.max() < 2e-2


def test_fp64_directional_derivative_matches_central_difference():
    Fm = F()
    p = wet_case(seed=6)
    steps = 30
    w = np.random.default_rng(9).standard_normal((steps, len(GAUGES)))
    s = Fm.Sim(p, precision=Fm.F64)
    g = s.adjoint(steps, GAUGES, w, n_checkpoints=3)
    v = np.random.default_rng(10).standard_normal(p.n.shape)
    eps = 1e-6

    def loss(n):
        t = Fm.Sim(p, precision=Fm.F64)
        t.set_manning(n)
        return float(np.sum(t.run_gauges(steps, GAUGES) * w))
    fd = (loss(p.n + eps * v) - loss(p.n - eps * v)) / (2 * eps)
    assert float(np.sum(g * v)) == pytest.approx(fd, rel=1e-6)


def test_autograd_function_gives_the_adjoint_gradient():
    import torch
    from paper_2204_10323_gb300.autograd import FloodRun
    Fm = F()
    p = wet_case(seed=7)
    s = Fm.Sim(p, precision=Fm.F64)
    n = torch.tensor(p.n, dtype=torch.float64, requires_grad=True)
    series = FloodRun.apply(n, s, GAUGES, 25, 4)
    obs = series.detach() + 0.01
    loss = ((series - obs) ** 2).sum()
    loss.backward()
    t = Fm.Sim(p, precision=Fm.F64)
    ref = t.adjoint(25, GAUGES, (2 * (series - obs)).detach().numpy(), n_checkpoints=25)
    np.testing.assert_allclose(n.grad.numpy(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    # the simulator ends where a plain 25-step run ends
    u = Fm.Sim(p, precision=Fm.F64)
    u.step(25)
    assert np.array_equal(s.read(Fm.FIELD_H), u.read(Fm.FIELD_H))


def test_calibration_1024_fp32_adjoint_vs_fp64_finite_differences():
    """Full-size calibration case: 1024^2, 16 gauges, 2000 steps, 40 snapshots."""
    Fm = F()
    steps = 2000
    truth = inputs.c5_calibration(truth=True, steps=steps)
    p = inputs.c5_calibration(truth=False, steps=steps)
    g = p.gauges
    obs = Fm.Sim(truth).run_gauges(steps, g)
    s = Fm.Sim(p)
    series = s.run_gauges(steps, g)
    seed = 2.0 * (series - obs)
    s2 = Fm.Sim(p)
    grad = s2.adjoint(steps, g, seed, n_checkpoints=40).astype(np.float64)
    assert s2.adjoint_forward_steps() == closed_cost(steps, 40) == 5097
    assert np.isfinite(grad).all()
    # 20 random cells among those the loss is sensitive to
    cand = np.argwhere(np.abs(grad) > 1e-2 * np.abs(grad).max())
    pick = cand[np.random.default_rng(11).choice(len(cand), size=min(20, len(cand)), replace=False)]
    p64 = Fm.Sim(p, precision=Fm.F64)
    base_state = p64.state()
    obs64 = obs

    def loss(n):
        p64.write_state(*base_state)
        p64.set_clock(0.0, 0, 0.0)
        p64.set_manning(n)
        h = p64.run_gauges(steps, g)
        return float(np.sum((h - obs64) ** 2))
    fd, ad = [], []
    for (j, i) in pick:
        eps = 1e-3 * p.n[j, i]
        a = p.n.copy()
        a[j, i] += eps
        b = p.n.copy()
        b[j, i] -= eps
        fd.append((loss(a) - loss(b)) / (2 * eps))
        ad.append(grad[j, i])
    fd, ad = np.array(fd), np.array(ad)
    cos = float(np.sum(fd * ad) / (np.linalg.norm(fd) * np.linalg.norm(ad)))
    assert cos > 0.999
    assert np.median(np.abs(ad - fd) / np.abs(fd)) < 1e-2
