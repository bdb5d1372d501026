"""Differentiable time stepping: a torch.autograd.Function around the C ABI.

The forward pass advances the state with CFL steps (dt on the device) and records dt and the LF
coefficients of every stage; the backward pass applies the hand-written adjoint step
(hweno_adjoint_step_stages) in reverse, with the derivative taken at the recorded dt and alphas.
Two ways to have the stage inputs every adjoint step needs:
  * checkpoints (the default): the state is saved every `every` steps; within a segment the
    states and the two stage inputs of every step are recomputed from its checkpoint by replaying
    the recorded steps (one extra forward step per step, memory of `every` steps);
  * keep_stages: the forward pass keeps the input and both stage inputs of every step (three states
    per step in device memory: 0.3 GB per step of 2D Euler at 1024^2), and the backward pass is
    adjoint steps alone.
Both give the same gradient bit for bit.
"""
from __future__ import annotations

import numpy as np
import torch

from .solver import Solver


class Rollout(torch.autograd.Function):
    """S0 -> state after nsteps steps.  Arguments: S0 (device tensor in the state layout), the
    Solver, nsteps, checkpoint interval, keep_stages (keep every step's stage inputs instead of
    checkpoints)."""

    @staticmethod
    def forward(ctx, S0: torch.Tensor, solver: Solver, nsteps: int, every: int, keep_stages: bool = False):
        every = max(1, int(every))
        with torch.cuda.stream(solver.stream):
            solver.state.copy_(S0.reshape(solver.state.shape))
        solver.set_time(0.0, 0.0)
        rec = torch.empty((nsteps, 7), dtype=torch.float64, device=solver.device)
        checkpoints, stages = [], None
        if keep_stages:
            stages = torch.empty((nsteps, 3) + tuple(solver.state.shape), dtype=solver.state.dtype,
                                 device=solver.device)
        for s in range(nsteps):
            if keep_stages:
                stages[s, 0].copy_(solver.state)
                solver.step_stages(stages[s, 1], stages[s, 2])
            else:
                if s % every == 0:
                    checkpoints.append(solver.state.clone())
                solver.step(0.0)
            solver.record(rec[s])
        solver.sync()
        ctx.solver, ctx.rec, ctx.checkpoints, ctx.every, ctx.nsteps = solver, rec, checkpoints, every, nsteps
        ctx.stages = stages
        ctx.dts = rec[:, 0].cpu().numpy()
        return solver.state.clone().reshape(S0.shape)

    @staticmethod
    def backward(ctx, lam_T: torch.Tensor):
        solver, rec, every, nsteps, dts = ctx.solver, ctx.rec, ctx.every, ctx.nsteps, ctx.dts
        lam = lam_T.contiguous().reshape(solver.state.shape).clone()
        if ctx.stages is not None:
            for s in range(nsteps - 1, -1, -1):
                St = ctx.stages[s]
                lam = solver.adjoint_step_stages(St[0], St[1], St[2], float(dts[s]), rec[s, 1:].contiguous(), lam)
            ctx.stages = None
            return lam.reshape(lam_T.shape), None, None, None, None
        nseg = (nsteps + every - 1) // every
        for seg in range(nseg - 1, -1, -1):
            s0, s1 = seg * every, min((seg + 1) * every, nsteps)
            # replay the segment from its checkpoint, keeping every step's input and stage inputs
            states = [(ctx.checkpoints[seg], torch.empty_like(solver.state), torch.empty_like(solver.state))]
            with torch.cuda.stream(solver.stream):
                solver.state.copy_(states[0][0])
            for s in range(s0, s1):
                Sn, S1, S2 = states[-1]
                solver.step_replay_stages(float(dts[s]), rec[s, 1:], S1, S2)
                if s < s1 - 1:
                    states.append((solver.state.clone(), torch.empty_like(solver.state), torch.empty_like(solver.state)))
            for s in range(s1 - 1, s0 - 1, -1):
                Sn, S1, S2 = states[s - s0]
                lam = solver.adjoint_step_stages(Sn, S1, S2, float(dts[s]), rec[s, 1:].contiguous(), lam)
        return lam.reshape(lam_T.shape), None, None, None, None


def rollout(S0: torch.Tensor, solver: Solver, nsteps: int, every: int = 20, keep_stages: bool = False) -> torch.Tensor:
    return Rollout.apply(S0, solver, nsteps, every, keep_stages)


def replay(S0: torch.Tensor, solver: Solver, dts: np.ndarray, rec: torch.Tensor) -> torch.Tensor:
    """The forward pass again with the recorded dts and alphas (no gradient)."""
    with torch.cuda.stream(solver.stream):
        solver.state.copy_(S0.reshape(solver.state.shape))
    for s in range(len(dts)):
        solver.step_replay(float(dts[s]), rec[s, 1:])
    solver.sync()
    return solver.state.clone()
