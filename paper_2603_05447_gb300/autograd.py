"""torch.autograd binding of the ramp gradient.

``ramp_infidelity(knots, problem)`` returns L = 1 - |<psi_t|psi(T)>|^2 after
the RK4 ramp with schedule ``knots`` as a differentiable torch scalar.  Both
the loss and its gradient come from the library: the forward pass runs the
ramp with a checkpoint tape (gpe_ramp_forward) and the discrete adjoint
(gpe_ramp_backward), which returns L and dL/dknots together; the backward
pass hands the stored gradient to autograd.  The knots tensor lives on the
host (float64); the states live on the GPU.
"""
from __future__ import annotations

import torch

from . import gpe


class RampProblem:
    """A ramp on an existing blend grid: initial state, target state, g, dt,
    number of steps, schedule duration and checkpoint interval K.

    ``psi0`` and ``target`` are device arrays in the compact layout of the
    grid (or any pointer-like accepted by gpe_state_load)."""

    def __init__(self, grid, dtype, psi0, target, g, dt, nsteps, T_ramp, K=64, t0=0.0):
        self.grid, self.dtype = grid, dtype
        self.state = gpe.gpe_state_create(grid, dtype)
        self.target = gpe.gpe_state_create(grid, dtype)
        self.start = gpe.gpe_state_create(grid, dtype)
        gpe.gpe_state_load(self.start, psi0, gpe.GPE_LAYOUT_COMPACT)
        gpe.gpe_state_load(self.target, target, gpe.GPE_LAYOUT_COMPACT)
        self.g, self.dt, self.nsteps, self.T_ramp, self.K, self.t0 = g, dt, nsteps, T_ramp, K, t0
        self.tape = None

    def params(self, knots):
        return gpe.real_params(self.g, self.dt, gpe.GPE_V_BLEND, [float(k) for k in knots], self.T_ramp)

    def forward(self, knots):
        """Run the ramp from the start state; returns (loss, gradient) from
        the library's adjoint."""
        if self.tape is not None:
            gpe.gpe_tape_destroy(self.tape)
            self.tape = None
        gpe.gpe_state_copy(self.state, self.start)
        self.tape = gpe.gpe_ramp_forward(self.state, self.params(knots), self.nsteps, self.t0, self.K)
        return gpe.gpe_ramp_backward(self.tape, self.target, len(knots))

    def close(self):
        if self.tape is not None:
            gpe.gpe_tape_destroy(self.tape)
            self.tape = None
        for h in (self.state, self.target, self.start):
            gpe.gpe_state_destroy(h)


class _RampInfidelity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, knots, problem):
        loss, grad = problem.forward(knots.detach().cpu().tolist())
        ctx.grad = torch.tensor(grad, dtype=torch.float64)
        return torch.tensor(loss, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        return ctx.grad * grad_out, None


def ramp_infidelity(knots: torch.Tensor, problem: RampProblem) -> torch.Tensor:
    return _RampInfidelity.apply(knots, problem)
