"""Ensembles: many uneven scenarios in one launch per step must give exactly
what each scenario gives alone (the same stream-kernel arithmetic, bit for
bit), for every launch shape, with and without graph replay."""
import numpy as np
import pytest

import inputs
from inputs import Problem
import oracle

pytestmark = pytest.mark.gpu


def F():
    import paper_2204_10323_gb300 as F
    return F


def scenarios():
    shapes = [(130, 70, 2), (257, 129, 6), (64, 300, 17), (500, 40, 18), (33, 17, 0)]
    out = []
    for nx, ny, seed in shapes:
        p = inputs.random_small(nx, ny, seed)
        r = lambda a: None if a is None else a.astype(np.float32).astype(np.float64)
        p = Problem(p.name, p.nx, p.ny, p.dx, r(p.z), r(p.n), p.sections, p.opts, h0=r(p.h0), qx0=r(p.qx0),
                    qy0=r(p.qy0))
        out.append(p)
    return out


@pytest.mark.parametrize("warps,rows,spg,graph", [(4, 64, 4, True), (2, 16, 8, True), (1, 128, 4, False),
                                                  (4, 7, 12, True)])
def test_ensemble_equals_members_alone(warps, rows, spg, graph):
    Fm = F()
    probs = scenarios()
    ens = Fm.Ensemble(probs)
    ens.set_launch(warps, rows, spg, use_graph=graph)
    ens.step(3)
    ens.step(spg * 2)
    ens.step(5)
    n = 3 + 2 * spg + 5
    for mb, p in zip(ens.members, probs):
        s = Fm.Sim(p, kernel=Fm.KERNEL_STREAM)
        s.step(n)
        for f in (Fm.FIELD_H, Fm.FIELD_QX, Fm.FIELD_QY):
            assert np.array_equal(mb.read(f), s.read(f)), (p.name, f)
        La, Lb = mb.ledger(), s.ledger()
        for k in ("t", "dt", "V_in", "V_out", "V_clip", "volume", "step"):
            assert La[k] == pytest.approx(Lb[k], rel=1e-12, abs=1e-12), (p.name, k)
    ens.close()


@pytest.mark.parametrize("K,rows,spg,graph", [(4, 16, 4, True), (2, 7, 8, True), (4, 64, 4, False),
                                              (1, 33, 4, True), (2, 300, 4, False), (8, 16, 8, True),
                                              (8, 40, 16, False)])
def test_tiled_ensemble_equals_members_alone(K, rows, spg, graph):
    """K steps per launch over every scenario's (chunk, strip) items give the
    bits of each scenario stepped alone by the single-step kernel."""
    Fm = F()
    probs = scenarios()
    for p in probs:
        p.opts.epoch_steps = max(4, K)
    ens = Fm.Ensemble(probs)
    ens.set_launch(2, rows, spg, use_graph=graph)
    ens.set_kernel(Fm.KERNEL_TILED, K)
    for n in (3, 2 * spg, 5, 1):           # partial launches, graph replays, epoch ends
        ens.step(n)
    n = 3 + 2 * spg + 5 + 1
    for mb, p in zip(ens.members, probs):
        s = Fm.Sim(p, kernel=Fm.KERNEL_STREAM)
        s.step(n)
        for f in (Fm.FIELD_H, Fm.FIELD_QX, Fm.FIELD_QY):
            assert np.array_equal(mb.read(f), s.read(f)), (p.name, f)
        La, Lb = mb.ledger(), s.ledger()
        for k in ("t", "dt", "V_in", "volume", "step", "h_max"):
            assert La[k] == pytest.approx(Lb[k], rel=1e-12, abs=1e-12), (p.name, k)
        # boundary outflow and clipped depth are summed per lane in float over
        # runs of at most 32 rows by the temporal-blocking kernel
        for k in ("V_out", "V_clip"):
            assert La[k] == pytest.approx(Lb[k], rel=1e-6, abs=1e-9), (p.name, k)
    ens.close()


@pytest.mark.parametrize("K,graph", [(4, True), (8, False)])
def test_tiled_ensemble_of_one_member_equals_it_alone(K, graph):
    """A single member: the members are launched in two groups of about equal
    cells, so the second group is empty and only the first one steps."""
    Fm = F()
    p = scenarios()[1]
    p.opts.epoch_steps = max(4, K)
    ens = Fm.Ensemble([p])
    ens.set_launch(2, 16, 8, use_graph=graph)
    ens.set_kernel(Fm.KERNEL_TILED, K)
    for n in (3, 16, 5):
        ens.step(n)
    s = Fm.Sim(p, kernel=Fm.KERNEL_STREAM)
    s.step(24)
    for f in (Fm.FIELD_H, Fm.FIELD_QX, Fm.FIELD_QY):
        assert np.array_equal(ens.members[0].read(f), s.read(f)), f
    assert ens.members[0].ledger()["step"] == 24
    s.close()
    ens.close()


def test_ensemble_set_kernel_rejects_bad_values():
    Fm = F()
    probs = scenarios()[:2]
    ens = Fm.Ensemble(probs)
    E = probs[0].opts.epoch_steps
    with pytest.raises(Fm.FloodError):
        ens.set_kernel(Fm.KERNEL_ROWS, 0)
    with pytest.raises(Fm.FloodError):
        ens.set_kernel(Fm.KERNEL_TILED, 5)
    if E % 3:
        with pytest.raises(Fm.FloodError):
            ens.set_kernel(Fm.KERNEL_TILED, 3)
    ens.set_kernel(Fm.KERNEL_TILED, 0)
    ens.step(E)
    ens.close()


def test_ensemble_member_matches_oracle():
    Fm = F()
    probs = scenarios()
    ens = Fm.Ensemble(probs)
    ens.set_launch(4, 64, 4)
    ens.step(100)
    p = probs[1]
    o = oracle.Oracle(p)
    o.run(100)
    assert np.abs(ens.members[1].read(Fm.FIELD_H).astype(np.float64) - o.h).max() < 1e-3
    ens.close()


def test_autotuner_picks_and_caches(tmp_path, monkeypatch):
    from paper_2204_10323_gb300 import autotune
    Fm = F()
    monkeypatch.setenv("FLOOD_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    ens = Fm.Ensemble(scenarios())
    cands = [(0, 4, 64, 4), (4, 2, 32, 8), (2, 2, 16, 4)]     # (K, warps, rows, steps per graph)
    r = autotune.tune_ensemble(ens, candidates=cands, trial_steps=8)
    assert not r["cached"] and len(r["trials"]) == 3 and tuple(r["shape"]) in cands
    r2 = autotune.tune_ensemble(ens)
    assert r2["cached"] and r2["shape"] == r["shape"]
    ens.close()


def test_autotuner_times_an_ensemble_on_its_own_stream(tmp_path, monkeypatch):
    """An ensemble created on a side stream: the trial events are recorded on that
    stream, so each trial measures the work it launched (about 0 ms otherwise)."""
    import torch
    from paper_2204_10323_gb300 import autotune
    Fm = F()
    monkeypatch.setenv("FLOOD_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    side = torch.cuda.Stream()
    ens = Fm.Ensemble(scenarios(), stream=side)
    assert ens.stream is side
    cands = [(0, 4, 64, 4), (4, 2, 32, 8)]
    r = autotune.tune_ensemble(ens, candidates=cands, trial_steps=64)
    # the events bracket the steps: a trial of 64 steps takes at least a few microseconds each
    assert all(t > 1e-3 for _, t in r["trials"]), r["trials"]
    ens.close()
