"""Gradients of an MPM rollout through the library's hand-written adjoint.

``rollout`` runs n steps with a checkpoint of the whole particle state every
``every`` steps (``mpm_save_state``); ``gradient`` walks the segments
backwards: each segment is recomputed from its checkpoint with every step's
state kept, then ``mpm_adjoint_step`` is applied step by step from the last
to the first.  Memory: n / every checkpoints plus ``every`` states.

``Rollout`` wraps both in a ``torch.autograd.Function``: inputs Young's
modulus E (a 0-d tensor) and the initial positions and velocities; outputs
the final positions and velocities, both in particle-id order.  Its backward
returns dL/dE, dL/dx0 and dL/dv0.  The adjoint covers Neo-Hookean contexts in
deterministic mode with block size 4 (the library refuses the others).
"""
from __future__ import annotations

import torch

from . import mpm

ADJ = 24   # adjoint record per particle: x(3) v(3) C(9) F(9)


def rollout(sim: "mpm.Simulation", nsteps: int, every: int):
    """Run nsteps; return the checkpoints taken before steps 0, every, 2 every, ..."""
    nbytes = sim.state_bytes()
    ckpts = []
    done = 0
    while done < nsteps:
        buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        sim.save_state(buf)
        ckpts.append(buf)
        k = min(every, nsteps - done)
        sim.step(k)
        done += k
    return ckpts


def gradient(sim: "mpm.Simulation", ckpts, nsteps: int, every: int, adj_final: torch.Tensor):
    """dL/d(initial state) (n, 24), dL/dE and dL/dphi (Drucker-Prager; phi in
    degrees, every particle's angle moved together), given dL/d(final state)."""
    nbytes = sim.state_bytes()
    adj_next = adj_final.contiguous().clone()
    adj_cur = torch.empty_like(adj_next)
    dE = dphi = 0.0
    for s in range(len(ckpts) - 1, -1, -1):
        k0 = s * every
        k = min(every, nsteps - k0)
        states = []
        sim.load_state(ckpts[s])
        for j in range(k):
            buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            sim.save_state(buf)
            states.append(buf)
            if j + 1 < k:
                sim.step(1)
        for j in range(k - 1, -1, -1):
            sim.load_state(states[j])
            e, ph = sim.adjoint_step(adj_next, adj_cur)
            dE += e
            dphi += ph
            adj_next, adj_cur = adj_cur, adj_next
    return adj_next, dE, dphi


class Rollout(torch.autograd.Function):
    """(E, x0, v0) -> (x_n, v_n) through nsteps of a context built by
    ``make_sim(E, x0, v0)``; checkpoints every ``every`` steps."""

    @staticmethod
    def forward(ctx, E, x0, v0, make_sim, nsteps: int, every: int):
        sim = make_sim(float(E), x0, v0)
        ckpts = rollout(sim, nsteps, every)
        out = sim.read_particles({"x": torch.empty_like(x0), "v": torch.empty_like(v0)})
        ctx.sim, ctx.ckpts, ctx.nsteps, ctx.every = sim, ckpts, nsteps, every
        return out["x"], out["v"]

    @staticmethod
    def backward(ctx, gx, gv):
        n = gx.shape[0]
        adj = torch.zeros(n, ADJ, dtype=torch.float32, device=gx.device)
        adj[:, 0:3] = gx
        if gv is not None:
            adj[:, 3:6] = gv
        g0, dE, _ = gradient(ctx.sim, ctx.ckpts, ctx.nsteps, ctx.every, adj)
        ctx.sim.close()
        return (torch.tensor(dE, dtype=torch.float64), g0[:, 0:3].clone(), g0[:, 3:6].clone(), None, None, None)
