"""Time-averaged rotor loads as a differentiable function of pitch and d0.

``rotor_objective(lat, pitch, d0, steps, avg_last)`` returns, per rotor, the
mean thrust F.a and torque M.a over the last ``avg_last`` of ``steps`` steps
from the lattice's current state (Sec. 2.2.2 forces, Sec. 3.2 time loop).
Its backward calls ``hl_grad`` with the incoming gradients as the objective
weights: for outputs (T, Q) and upstream gradients (gT, gQ) the objective is
J = sum_k gT_k T_k + gQ_k Q_k, and hl_grad returns dJ/dpitch and dJ/dd0 of
the discrete step with the cell sets held at their forward values.

The forward pass saves the state, runs the steps and leaves the lattice
advanced; the backward pass restores the saved state, re-runs the steps with
checkpoints inside hl_grad and leaves the lattice advanced again.
"""

from __future__ import annotations

import numpy as np


def _autograd_function():
    import torch

    class RotorObjective(torch.autograd.Function):
        @staticmethod
        def forward(ctx, pitch, d0, lat, steps, avg_last, ckpt_every):
            p = pitch.detach().to("cpu", torch.float64).numpy()
            for k in range(lat.nrot):
                lat.set_pitch(k, float(p[k]))
            lat.set_d0(d0.detach())
            state = lat.save_state()
            lat.forces(reset_avg=True)
            lat.step(int(steps - avg_last))
            lat.forces(reset_avg=True)
            lat.step(int(avg_last))
            _, Fa = lat.forces()
            _, Ma = lat.moments()
            a = lat.cfg.flow_axis
            ctx.lat, ctx.state = lat, state
            ctx.steps, ctx.avg_last, ctx.ckpt = int(steps), int(avg_last), int(ckpt_every)
            ctx.d0_shape = d0.shape
            T = torch.as_tensor(Fa[:, a].copy(), dtype=pitch.dtype)
            Q = torch.as_tensor(Ma[:, a].copy(), dtype=pitch.dtype)
            return T, Q

        @staticmethod
        def backward(ctx, gT, gQ):
            lat = ctx.lat
            lat.load_state(ctx.state)
            wT = np.zeros(lat.nrot) if gT is None else gT.detach().to("cpu", torch.float64).numpy()
            wQ = np.zeros(lat.nrot) if gQ is None else gQ.detach().to("cpu", torch.float64).numpy()
            _, gp, gd0 = lat.grad(ctx.steps, ctx.avg_last, wT, wQ, ckpt_every=ctx.ckpt,
                                  want_d0=ctx.needs_input_grad[1])
            gpitch = torch.as_tensor(gp, dtype=torch.float64)
            gd = None if gd0 is None else gd0.reshape(ctx.d0_shape)
            return gpitch, gd, None, None, None, None

    return RotorObjective


_FN = None


def rotor_objective(lat, pitch, d0, steps: int, avg_last: int, ckpt_every: int = 100):
    """(mean thrust (nrot,), mean torque (nrot,)) over the last avg_last of `steps`
    steps, differentiable in pitch (nrot,) and d0 (device tensor, one value per cell)."""
    global _FN
    if _FN is None:
        _FN = _autograd_function()
    return _FN.apply(pitch, d0, lat, steps, avg_last, ckpt_every)
