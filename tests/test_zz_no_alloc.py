"""GPU check of flood_volume_noalloc, the entry point that allocates nothing.

Callers that cannot allocate device memory where they need the stored water
volume (inside a CUDA-graph capture region, under their own memory pool, or
in hosts that forbid allocation after start-up) use this variant of the
volume reduction; its scratch is a fixed device array inside the library.
The test calls it through the C ABI on two different states in a row (the
second call reuses the scratch the first one left behind) and checks each
result against the volume the handle-based entry point reports in its ledger.
This file is collected last on purpose so that a run stopping at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

REL = 1e-12      # both sides sum the same float32 depths in double precision; only the order differs


def test_volume_noalloc_matches_ledger_twice():
    import torch
    import paper_2204_10323_gb300 as F

    torch.cuda.set_device(0)
    p = inputs.c2_fractal(nx=700, ny=530, steps=100)
    p.h0 = inputs.wet_start(p.z, p.dx, 0.4)
    sim = F.Sim(p, precision=F.F32)
    depth = torch.empty((p.ny, p.nx), dtype=torch.float32, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    expect = []
    for call in range(2):
        sim.step(17 if call == 0 else 29)
        expect.append(sim.ledger()["volume"])
        F.flood_read(sim.h, F.FIELD_H, C.c_void_p(depth.data_ptr()), depth.numel() * 4, 1)
        F.flood_volume_noalloc(C.c_void_p(depth.data_ptr()), p.nx, p.ny, p.nx, F.F32, p.dx,
                               C.c_void_p(out.data_ptr() + 8 * call), None)
        torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert expect[0] != expect[1]
    for k in range(2):
        assert got[k] == pytest.approx(expect[k], rel=REL)
    sim.close()


def test_volume_noalloc_rejects_too_many_rows():
    import torch
    import paper_2204_10323_gb300 as F

    buf = torch.zeros(4, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = F.lib().flood_volume_noalloc(C.c_void_p(buf.data_ptr()), 1, 65537, 1, F.F32, 1.0,
                                      C.c_void_p(out.data_ptr()), None)
    assert st == F.ERR_ARG
    assert "65536" in F.flood_last_error(None)
