"""torch.autograd wrapper of the flood model: gauge depths as a differentiable
function of the per-cell Manning field.

``FloodRun.apply(n, sim, gauges, n_steps, n_checkpoints)`` runs ``n_steps``
steps of ``sim`` from its current state with Manning field ``n`` and returns
the depth at each gauge after every step, an (n_steps, G) float64 tensor.
Its backward pass calls ``flood_adjoint`` (binomial checkpointing with
``n_checkpoints`` device snapshots) from the same starting state and returns
dL/dn.  The time-step schedule is held fixed (it is chosen by the forward
run).  After forward and backward the simulator holds the end state of the
forward run, as after a plain run.
"""
from __future__ import annotations

import numpy as np
import torch


def _to_numpy(t: torch.Tensor, dtype) -> np.ndarray:
    return np.ascontiguousarray(t.detach().to("cpu").numpy(), dtype)


class FloodRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, n_field, sim, gauges, n_steps: int, n_checkpoints: int = 40):
        h0, qx0, qy0 = sim.state()
        clock0 = sim.ledger()
        sim.set_manning(_to_numpy(n_field, sim.dtype))
        series = sim.run_gauges(int(n_steps), np.asarray(gauges))
        ctx.sim = sim
        ctx.gauges = np.asarray(gauges)
        ctx.n_steps = int(n_steps)
        ctx.n_checkpoints = int(n_checkpoints)
        ctx.start = (h0, qx0, qy0, clock0)
        ctx.n_dtype, ctx.n_device = n_field.dtype, n_field.device
        return torch.from_numpy(series)

    @staticmethod
    def backward(ctx, grad_series):
        sim = ctx.sim
        h0, qx0, qy0, c0 = ctx.start
        h1, qx1, qy1 = sim.state()
        c1 = sim.ledger()
        sim.write_state(h0, qx0, qy0)
        sim.set_clock(c0["t"], int(c0["step"]), c0["dt"], c0["V_in"], c0["V_out"], c0["V_clip"])
        seed = _to_numpy(grad_series, np.float64)
        g = sim.adjoint(ctx.n_steps, ctx.gauges, seed, ctx.n_checkpoints)
        sim.write_state(h1, qx1, qy1)
        sim.set_clock(c1["t"], int(c1["step"]), c1["dt"], c1["V_in"], c1["V_out"], c1["V_clip"])
        grad_n = torch.from_numpy(np.asarray(g)).to(dtype=ctx.n_dtype, device=ctx.n_device)
        return grad_n, None, None, None, None
