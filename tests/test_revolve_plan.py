"""The adjoint's checkpoint schedule (binomial checkpointing, "revolve") run on
the host through flood_revolve_plan: the same recursion flood_adjoint drives
on the device, without a grid or a GPU.

Pins: the forward steps it replays equal the optimum of the checkpointing
recurrence F(l, s) = min_j [j + F(l - j, s - 1) + F(j, s)], F(1, s) = 0,
F(l, 0) = l (l - 1) / 2 (l steps to reverse, s free slots besides the start
state's), solved here by brute force, and Griewank's closed form r l -
C(c + r, c + 1) (c = s + 1 slots, r the least integer with C(c + r, c) >= l);
every step is reversed once, from the last to the first; every restore
reads a snapshot that holds the step it claims (the library checks that and
fails otherwise); replay launches of up to four steps never cross an epoch end.
"""
import functools
import math

import pytest


def F():
    import paper_2204_10323_gb300 as F
    return F


@functools.lru_cache(maxsize=None)
def optimum(l, s):
    """Fewest forward steps to reverse l steps from a stored start with s free slots."""
    if l <= 1:
        return 0
    if s == 0:
        return l * (l - 1) // 2
    return min(j + optimum(l - j, s - 1) + optimum(j, s) for j in range(1, l))


def closed_form(l, c):
    if l <= 1:
        return 0
    r = 0
    while math.comb(c + r, c) < l:
        r += 1
    return r * l - math.comb(c + r, c + 1)


def test_closed_form_is_the_recurrence_optimum():
    for l in range(1, 61):
        for c in range(1, 13):
            assert closed_form(l, c) == optimum(l, c - 1), (l, c)


@pytest.mark.parametrize("c", [1, 2, 3, 5, 8, 13])
def test_schedule_replays_the_optimum_and_reverses_in_order(c):
    Fm = F()
    for l in range(1, 61):
        p = Fm.revolve_plan(l, c)
        assert p["in_order"], (l, c)
        assert p["forward_steps"] == optimum(l, min(c, l) - 1), (l, c)
        assert p["replay_launches"] == p["forward_steps"]        # one step per launch


def test_paper_scale_sweep():
    """2000 steps with 40 snapshots: r = 3 repetitions, 3 * 2000 - C(43, 41) = 5097."""
    p = F().revolve_plan(2000, 40)
    assert p["in_order"]
    assert p["forward_steps"] == 5097 == closed_form(2000, 40)


@pytest.mark.parametrize("E,start", [(16, 0), (16, 5), (4, 3), (1, 0), (7, 2)])
def test_multi_step_replays_keep_the_count_and_stop_at_epoch_ends(E, start):
    Fm = F()
    for l, c in [(2000, 40), (300, 6), (97, 3), (45, 22), (33, 1)]:
        one = Fm.revolve_plan(l, c, E, start, 1)
        four = Fm.revolve_plan(l, c, E, start, 4)
        assert one["in_order"] and four["in_order"]
        assert four["forward_steps"] == one["forward_steps"] == closed_form(l, min(c, l))
        assert math.ceil(four["forward_steps"] / 4) <= four["replay_launches"] <= four["forward_steps"]
        if E == 1:                      # every step ends an epoch: single-step launches only
            assert four["replay_launches"] == four["forward_steps"]
    # 2000 steps in epochs of 16 from an epoch start: most replays run four steps at a time
    assert Fm.revolve_plan(2000, 40, 16, 0, 4)["replay_launches"] < 0.6 * 5097


def test_snapshot_count_above_the_steps_keeps_every_state():
    p = F().revolve_plan(45, 1000)
    assert p["in_order"] and p["forward_steps"] == 44


@pytest.mark.parametrize("args", [(0, 4, 16, 0, 1), (10, 0, 16, 0, 1), (10, 4, 0, 0, 1), (10, 4, 16, -1, 1),
                                  (10, 4, 16, 0, 0), (2_000_000, 4, 16, 0, 1)])
def test_plan_rejects_bad_arguments(args):
    Fm = F()
    with pytest.raises(Fm.FloodError):
        Fm.revolve_plan(*args)
