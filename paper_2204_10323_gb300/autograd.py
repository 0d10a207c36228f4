"""torch.autograd wrapper of the flood model: gauge depths as a differentiable
function of the per-cell Manning field.

``FloodRun.apply(n, sim, gauges, n_steps, n_checkpoints)`` runs ``n_steps``
steps of ``sim`` from its current state with Manning field ``n`` and returns
the depth at each gauge after every step, an (n_steps, G) float64 tensor on
``n``'s device.  Its backward pass calls ``flood_adjoint`` (binomial
checkpointing with ``n_checkpoints`` device snapshots) from the same starting
state and returns dL/dn.  The time-step schedule is held fixed (it is chosen
by the forward run).  After forward and backward the simulator holds the end
state of the forward run, as after a plain run.

The starting and end states are kept in device tensors (flood_read and
flood_write_state on device memory); only the 9-value ledgers and the gauge
seeds of the loss cross to the host.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch


def _state_to_device(sim):
    """The handle's (h, qx, qy) copied into new CUDA tensors of its precision."""
    import paper_2204_10323_gb300 as F
    dt = torch.float32 if sim.precision == F.F32 else torch.float64
    shapes = ((F.FIELD_H, (sim.ny, sim.nx)), (F.FIELD_QX, (sim.ny, sim.nx + 1)), (F.FIELD_QY, (sim.ny + 1, sim.nx)))
    out = []
    for field, shape in shapes:
        t = torch.empty(shape, dtype=dt, device="cuda")
        F.flood_read(sim.h, field, C.c_void_p(t.data_ptr()), t.numel() * t.element_size(), 1)
        out.append(t)
    return out


def _restore(sim, state, clock):
    h, qx, qy = state
    sim.write_state(h, qx, qy)                  # device input: taken as it is, no host round trip
    sim.set_clock(clock["t"], int(clock["step"]), clock["dt"], clock["V_in"], clock["V_out"], clock["V_clip"])


class FloodRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, n_field, sim, gauges, n_steps: int, n_checkpoints: int = 40):
        import paper_2204_10323_gb300 as F
        start = _state_to_device(sim)
        clock0 = sim.ledger()
        ndt = torch.float32 if sim.precision == F.F32 else torch.float64
        n_dev = n_field.detach().to(device="cuda", dtype=ndt).contiguous()
        sim.set_manning(n_dev)
        gauges = np.asarray(gauges)
        series = torch.empty((int(n_steps), len(gauges)), dtype=torch.float64, device="cuda")
        sim.run_gauges(int(n_steps), gauges, out=series)
        ctx.sim = sim
        ctx.gauges = gauges
        ctx.n_steps = int(n_steps)
        ctx.n_checkpoints = int(n_checkpoints)
        ctx.start = (start, clock0)
        ctx.n_dtype, ctx.n_device = n_field.dtype, n_field.device
        return series.to(n_field.device)

    @staticmethod
    def backward(ctx, grad_series):
        import paper_2204_10323_gb300 as F
        sim = ctx.sim
        start, c0 = ctx.start
        end = _state_to_device(sim)
        c1 = sim.ledger()
        _restore(sim, start, c0)
        seed = np.ascontiguousarray(grad_series.detach().to("cpu").numpy(), np.float64)   # (n_steps, G) doubles
        cells = np.ascontiguousarray(ctx.gauges[:, 1].astype(np.int64) * sim.nx + ctx.gauges[:, 0], np.int64)
        ndt = torch.float32 if sim.precision == F.F32 else torch.float64
        gn = torch.empty((sim.ny, sim.nx), dtype=ndt, device="cuda")
        F.flood_adjoint(sim.h, ctx.n_steps, cells.ctypes.data_as(C.POINTER(C.c_int64)), cells.size,
                        seed.ctypes.data_as(C.POINTER(C.c_double)), ctx.n_checkpoints, C.c_void_p(gn.data_ptr()),
                        None, 1)
        _restore(sim, end, c1)
        grad_n = gn.to(dtype=ctx.n_dtype, device=ctx.n_device)
        return grad_n, None, None, None, None
