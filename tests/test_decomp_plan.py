"""Row-strip decomposition on the host (Methods, "TPU Implementation"; Results,
"Scaling on TPU": 1 x N strips): the C library's row split and halo-copy list,
its ledger combine, and an exchange between two gloo ranks on the CPU that
follows the copy list with point-to-point messages and reduces h_max and the
ledger terms with all-reduces.  No GPU work: flood_decomp_plan and
flood_decomp_combine_ledgers touch no device."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FIELDS = (0, 1, 2)          # FLOOD_FIELD_H, _QX, _QY


def F():
    import paper_2204_10323_gb300 as F
    return F


def global_state(nx, ny, seed):
    rng = np.random.default_rng(seed)
    return {0: rng.uniform(0, 2, (ny, nx)), 1: rng.uniform(-1, 1, (ny, nx + 1)), 2: rng.uniform(-1, 1, (ny + 1, nx))}


def local_arrays(g, a, b):
    """A part's stored rows [a, b) (face rows [a, b] for qy), halo rows poisoned."""
    return {0: g[0][a:b].copy(), 1: g[1][a:b].copy(), 2: g[2][a:b + 1].copy()}


def poison(loc, y0, y1, a):
    for f in FIELDS:
        keep = np.zeros(loc[f].shape[0], bool)
        keep[y0 - a:y1 - a + (1 if f == 2 else 0)] = True     # own rows; qy: own face rows [y0, y1]
        loc[f][~keep] = np.nan


@pytest.mark.parametrize("ny,n_parts,halo", [(20, 3, 2), (128, 4, 4), (129, 4, 3), (8, 2, 4), (40, 40, 1),
                                             (1000, 7, 16), (5, 1, 3)])
def test_plan_rows_partition_the_grid(ny, n_parts, halo):
    rows, copies = F().flood_decomp_plan(ny, n_parts, halo)
    assert rows[0, 0] == 0 and rows[-1, 1] == ny
    assert np.array_equal(rows[1:, 0], rows[:-1, 1])                  # own rows tile [0, ny)
    assert (rows[:, 1] - rows[:, 0] >= min(halo, ny)).all() or n_parts == 1
    assert np.array_equal(rows[:, 0], [r * ny // n_parts for r in range(n_parts)])
    assert np.array_equal(rows[:, 2], np.maximum(rows[:, 0] - halo * (np.arange(n_parts) > 0), 0))
    assert np.array_equal(rows[:, 3], np.where(np.arange(n_parts) < n_parts - 1, rows[:, 1] + halo, ny))
    assert len(copies) == 6 * (n_parts - 1)


@pytest.mark.parametrize("nx,ny,n_parts,halo", [(7, 20, 3, 2), (5, 128, 4, 4), (3, 129, 4, 3), (9, 8, 2, 4),
                                                (4, 1000, 7, 16)])
def test_plan_copies_rebuild_every_halo_row_from_own_rows(nx, ny, n_parts, halo):
    """Applying the copy list to parts whose halo rows are poisoned gives every
    part the whole grid's rows [a, b); every source row is one its part owns
    (qy: a face row of [y0, y1], which a part computes exactly)."""
    rows, copies = F().flood_decomp_plan(ny, n_parts, halo)
    g = global_state(nx, ny, 1)
    loc = []
    for y0, y1, a, b in rows:
        L = local_arrays(g, a, b)
        poison(L, y0, y1, a)
        loc.append(L)
    for field, sp, sr, dp, dr, n in copies:
        y0, y1, a, _ = rows[sp]
        top = y1 + (1 if field == 2 else 0)
        assert y0 <= a + sr and a + sr + n <= top, "copy source outside the source part's exact rows"
        loc[dp][field][dr:dr + n] = loc[sp][field][sr:sr + n]
    for (y0, y1, a, b), L in zip(rows, loc):
        ref = local_arrays(g, a, b)
        for f in FIELDS:
            assert np.array_equal(L[f], ref[f]), (f, a, b)


def test_plan_rejects_bad_splits():
    Fm = F()
    for args in [(10, 4, 3), (10, 0, 1), (10, 2, 0), (3, 4, 1)]:
        with pytest.raises(Fm.FloodError) as e:
            Fm.flood_decomp_plan(*args)
        assert e.value.status == Fm.ERR_ARG


def test_combine_ledgers():
    Fm = F()
    # t, dt, V_in, V_out, V_clip, volume, h_max, step, cfl
    parts = np.array([[10.0, 0.5, 7.0, 1.0, 0.25, 100.0, 2.0, 20, 0],
                      [10.0, 0.5, 0.0, 2.0, 0.5, 50.0, 3.5, 20, 0],
                      [10.0, 0.5, 0.0, 0.5, 0.0, 25.0, 1.0, 20, 0]])
    out = Fm.flood_decomp_combine_ledgers(parts)
    assert out.tolist() == [10.0, 0.5, 7.0, 3.5, 0.75, 175.0, 3.5, 20, 0]
    parts[2, 7] = 21                                      # a part one step ahead
    with pytest.raises(Fm.FloodError) as e:
        Fm.flood_decomp_combine_ledgers(parts)
    assert e.value.status == Fm.ERR_STATE


# ---------------------------------------------------------------- two CPU ranks
def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import inputs
    import oracle
    import paper_2204_10323_gb300 as Fm
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        p = inputs.random_small(23, 31, 2)
        nx, ny, halo = p.nx, p.ny, 4
        rows, copies = Fm.flood_decomp_plan(ny, world, halo)
        y0, y1, a, b = (int(v) for v in rows[rank])
        g = {0: p.h0, 1: p.qx0, 2: p.qy0}
        loc = local_arrays(g, a, b)
        poison(loc, y0, y1, a)
        # halo exchange along the copy list: sends of own rows, receives into halo rows
        reqs, bufs = [], []
        for field, sp, sr, dp, dr, n in copies:
            if sp == rank:
                t = torch.from_numpy(np.ascontiguousarray(loc[field][sr:sr + n]))
                reqs.append(dist.isend(t, dst=dp, tag=field))
            if dp == rank:
                t = torch.empty((n, loc[field].shape[1]), dtype=torch.float64)
                bufs.append((field, dr, n, t))
                reqs.append(dist.irecv(t, src=sp, tag=field))
        for r in reqs:
            r.wait()
        for field, dr, n, t in bufs:
            loc[field][dr:dr + n] = t.numpy()
        ref = local_arrays(g, a, b)
        exchanged = all(np.array_equal(loc[f], ref[f]) for f in FIELDS)
        # epoch start: the largest own-row depth of the ranks
        own_h = loc[0][y0 - a:y1 - a]
        hmax = torch.tensor([own_h.max()], dtype=torch.float64)
        dist.all_reduce(hmax, op=dist.ReduceOp.MAX)
        # the ranks' own ledger terms combined by the library's rule
        mine = np.array([3.0, 0.25, 5.0 if rank == 0 else 0.0, 0.1 * (rank + 1), 0.0,
                         float(own_h.sum()) * p.dx * p.dx, float(own_h.max()), 12, 0], np.float64)
        allL = [torch.zeros(9, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(allL, torch.from_numpy(mine))
        whole = Fm.flood_decomp_combine_ledgers(np.stack([t.numpy() for t in allL]))
        out.put((rank, exchanged, float(hmax.item()), whole.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_exchange_halos_and_reduce():
    import inputs
    import oracle
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(300)
        assert pr.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    p = inputs.random_small(23, 31, 2)
    o = oracle.Oracle(p)
    for rank, exchanged, hmax, whole in got:
        assert exchanged, rank
        assert hmax == p.h0.max()                          # the whole grid's maximum, exactly
        # the time-step rule on the reduced maximum is the rule on the whole grid
        one = oracle.Oracle(inputs.Problem("one", 1, 1, p.dx, np.zeros((1, 1)), np.full((1, 1), 0.03), [], p.opts,
                                           h0=np.full((1, 1), hmax)))
        assert one.dt() == o.dt()
        assert whole[2] == 5.0 and whole[3] == pytest.approx(0.3) and whole[7] == 12
        assert whole[5] == pytest.approx(o.volume(), rel=1e-12)
        assert whole[6] == p.h0.max()
