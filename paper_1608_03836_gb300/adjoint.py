"""Receiver traces as a differentiable function of the initial pressure and c^2.

``receiver_traces(mesh, p0, c2q, dt, nsteps)`` runs nsteps LSRK(5,4) steps of
the WADG solver from Q = (p0, 0, 0, 0), res = 0, with the mesh's point sources
and receivers, and returns the receiver pressures after every step,
``traces[n, s, r]``.  It is a torch.autograd.Function: the backward pass runs
the library's discrete adjoint (wadg_step_adjoint, wadg_receivers_adjoint),
giving exact gradients of any scalar function of the traces with respect to
the nodal initial pressure and the c^2 values at the volume quadrature points.

Memory: the forward pass keeps Q every ``checkpoint`` steps; the
backward pass makes one library call per segment (wadg_segment_adjoint),
which recomputes the segment forward once, recording the 5 stage factors of
every step (5 K S Nq values per step), then reverses it step by step.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api as W


def _full_Q(mesh, p0):
    Q = torch.zeros((4, mesh.K, mesh.S, mesh.Np), dtype=mesh.dtype, device="cuda")
    Q[0] = p0.to(mesh.dtype)
    return Q


class _ReceiverTraces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, p0, c2q, mesh, dt, nsteps, checkpoint, t0):
        W.wadg_set_operators(mesh, mesh.precision, mesh.S, mesh.tau_p, mesh.tau_u, c2q.detach().cpu().numpy())
        Q = _full_Q(mesh, p0.detach())
        R = torch.zeros_like(Q)
        traces = torch.zeros((nsteps, mesh.S, mesh.R), dtype=mesh.dtype, device="cuda")
        checkpoints = []
        for n in range(nsteps):
            if n % checkpoint == 0:
                checkpoints.append(Q.clone())
            W.wadg_step_record(mesh, Q, R, t0 + n * dt, dt, None, traces[n])
        ctx.mesh, ctx.dt, ctx.nsteps, ctx.checkpoint, ctx.t0 = mesh, dt, nsteps, checkpoint, t0
        ctx.checkpoints = checkpoints
        return traces

    @staticmethod
    def backward(ctx, g):
        mesh, dt, nsteps, cp, t0 = ctx.mesh, ctx.dt, ctx.nsteps, ctx.checkpoint, ctx.t0
        g = g.to(mesh.dtype).contiguous()
        lamQ = torch.zeros((4, mesh.K, mesh.S, mesh.Np), dtype=mesh.dtype, device="cuda")
        lamR = torch.zeros_like(lamQ)
        dc2 = torch.zeros((mesh.K, mesh.Nq), dtype=torch.float64, device="cuda")
        nseg = len(ctx.checkpoints)
        for seg in reversed(range(nseg)):
            n0, n1 = seg * cp, min(nsteps, (seg + 1) * cp)
            Q = ctx.checkpoints[seg].clone()
            R = torch.zeros_like(Q)  # a step's first stage (a_1 = 0) does not read res
            ys = torch.empty((n1 - n0, 5, mesh.K, mesh.S, mesh.Nq), dtype=mesh.dtype, device="cuda")
            # one library call: recompute with recording, then the reverse steps
            W.wadg_segment_adjoint(mesh, Q, R, t0 + n0 * dt, dt, n1 - n0, g[n0:n1] if mesh.R > 0 else None,
                                   lamQ, lamR, ys, dc2)
            del ys
        grad_p0 = lamQ[0].clone()
        return grad_p0, dc2, None, None, None, None, None


def receiver_traces(mesh, p0, c2q, dt: float, nsteps: int, checkpoint: int = 20, t0: float = 0.0):
    """Differentiable traces[n, s, r] (see the module docstring).

    p0: CUDA tensor (K, S, Np) of nodal initial pressures; c2q: CUDA float64
    tensor (K, Nq) of c^2 at the volume quadrature points.  The mesh must have
    operators, sources and receivers set; its precision sets the arithmetic.
    """
    return _ReceiverTraces.apply(p0, c2q, mesh, float(dt), int(nsteps), int(checkpoint), float(t0))
