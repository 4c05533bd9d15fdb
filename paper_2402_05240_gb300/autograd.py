"""torch.autograd glue for the VL+CT step (the adjoint itself is mhd_adjoint_step).

MHDStep: one step at fixed dt; forward = mhd_step on a copy, backward =
mhd_adjoint_step.  rollout(): n steps with step-level checkpointing: the
forward keeps the state every ``checkpoint_every`` steps; the backward
recomputes each segment from its checkpoint (with the recorded dt sequence)
and runs the adjoint steps of the segment in reverse, so at most
``checkpoint_every + n / checkpoint_every`` states are held at once.

When ``dts`` is not given, the forward takes dt from the device CFL
reduction of each step (Step 1) and records it.  By default the derivative
treats that sequence as constant; with ``dt_grad=True`` each step's dt is
differentiated as the function of its start state that it is
(mhd_adjoint_step_cfl), so the gradient is that of the rollout as run.
"""
from __future__ import annotations

import torch

from . import mhd as _mhd


class MHDStep(torch.autograd.Function):
    """U^{n+1} = step(U^n) at fixed dt."""

    @staticmethod
    def forward(ctx, U, dt, sim):
        out = U.detach().contiguous().clone()
        sim.step(out, float(dt))
        ctx.save_for_backward(U.detach())
        ctx.dt = float(dt)
        ctx.sim = sim
        return out

    @staticmethod
    def backward(ctx, g):
        (U,) = ctx.saved_tensors
        gU = ctx.sim.adjoint_step(U.contiguous(), ctx.dt, g.contiguous())
        return gU, None, None


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, sim, nsteps, dts, k, dt_grad=False):
        U = U0.detach().contiguous().clone()
        ckpt = {0: U.clone()}
        dts_used = []
        for s in range(nsteps):
            if dts is None:
                dt_dev = torch.zeros(1, dtype=torch.float64, device=U.device)
                _mhd.mhd_run(sim.ctx, U, 1, dt_dev)
                dts_used.append(float(dt_dev.item()))
            else:
                sim.step(U, float(dts[s]))
                dts_used.append(float(dts[s]))
            if (s + 1) % k == 0 and s + 1 < nsteps:
                ckpt[s + 1] = U.clone()
        ctx.sim = sim
        ctx.k = k
        ctx.nsteps = nsteps
        ctx.dts = dts_used
        ctx.ckpt = ckpt
        ctx.dt_grad = bool(dt_grad) and dts is None
        return U

    @staticmethod
    def backward(ctx, g):
        sim, k, n, dts = ctx.sim, ctx.k, ctx.nsteps, ctx.dts
        g = g.contiguous().clone()
        starts = sorted(ctx.ckpt.keys())
        for a in reversed(starts):
            b = min(a + k, n)
            # recompute the states of the segment [a, b)
            states = [ctx.ckpt[a]]
            U = ctx.ckpt[a].clone()
            for s in range(a, b - 1):
                sim.step(U, dts[s])
                states.append(U.clone())
            for s in range(b - 1, a - 1, -1):
                if ctx.dt_grad:
                    g, dt, _ = sim.adjoint_step_cfl(states[s - a], g)
                    if dt != dts[s]:
                        raise RuntimeError(f"step {s}: recomputed CFL dt {dt!r} differs from the forward's {dts[s]!r}")
                else:
                    g = sim.adjoint_step(states[s - a], dts[s], g)
            del states
        ctx.ckpt = None
        return g, None, None, None, None, None


def rollout(sim, U0: torch.Tensor, nsteps: int, dts=None, checkpoint_every: int | None = None,
            dt_grad: bool = False) -> torch.Tensor:
    """``nsteps`` VL+CT steps from U0, differentiable with respect to U0.

    dts: fixed dt sequence (else the device CFL dt of each step, recorded).
    checkpoint_every: segment length k of the step-level checkpointing
    (default: no intermediate checkpoints, one segment of nsteps).
    dt_grad: with dts=None, also differentiate each CFL dt through its
    start state (else the recorded dts are constants of the derivative).
    Returns U^{n}; ``rollout.last_dts`` is not kept: pass ``dts`` to control them.
    """
    k = int(checkpoint_every) if checkpoint_every else max(int(nsteps), 1)
    return _Rollout.apply(U0, sim, int(nsteps), None if dts is None else [float(x) for x in dts], k, bool(dt_grad))


def magnetic_energy(U: torch.Tensor, dV: float) -> torch.Tensor:
    """L = sum over cells of |B_cc|^2 / 2 * dV, with B_cc the face mean."""
    bx = 0.5 * (U[5] + torch.roll(U[5], 1, dims=2))
    by = 0.5 * (U[6] + torch.roll(U[6], 1, dims=1))
    bz = 0.5 * (U[7] + torch.roll(U[7], 1, dims=0))
    return 0.5 * dV * torch.sum(bx * bx + by * by + bz * bz)


def conserved_from(rho, vel, pres, bface, gamma: float) -> torch.Tensor:
    """Differentiable state assembly U(rho, v, P, B_face) (Sec. 2.1): used to
    take gradients with respect to the velocity at fixed rho, P and with
    respect to the face field."""
    bx, by, bz = bface
    bcx = 0.5 * (bx + torch.roll(bx, 1, dims=2))
    bcy = 0.5 * (by + torch.roll(by, 1, dims=1))
    bcz = 0.5 * (bz + torch.roll(bz, 1, dims=0))
    vx, vy, vz = vel
    E = pres / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) + 0.5 * (bcx * bcx + bcy * bcy + bcz * bcz)
    return torch.stack([rho, rho * vx, rho * vy, rho * vz, E, bx, by, bz]).contiguous()
