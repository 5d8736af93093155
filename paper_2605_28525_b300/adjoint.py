"""Gradients of an MPM rollout through the library's hand-written adjoint.

``rollout`` runs n steps with a checkpoint of the whole particle state every
``every`` steps (``mpm_save_state``); ``gradient`` walks the segments
backwards: each segment is recomputed from its checkpoint with every step's
state kept, then ``mpm_adjoint_step`` is applied step by step from the last
to the first.  Memory: n / every checkpoints plus ``every`` states.

``Rollout`` wraps both in a ``torch.autograd.Function``: inputs Young's
modulus E and the friction angle phi (0-d tensors, phi in degrees, one angle
for every particle) and the initial positions and velocities; outputs the
final positions and velocities, both in particle-id order.  Its backward
returns dL/dE, dL/dphi, dL/dx0 and dL/dv0.  The adjoint covers Neo-Hookean
and Drucker-Prager contexts in deterministic mode with block size 4 (the
library refuses the others).
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
    """(E, phi, x0, v0) -> (x_n, v_n) through nsteps of a context built by
    ``make_sim(E, phi, x0, v0)``; checkpoints every ``every`` steps.  E and
    phi are 0-d tensors (phi in degrees, one angle for every particle)."""

    @staticmethod
    def forward(ctx, E, phi, x0, v0, make_sim, nsteps: int, every: int):
        sim = make_sim(float(E), float(phi), x0, v0)
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
        g0, dE, dphi = gradient(ctx.sim, ctx.ckpts, ctx.nsteps, ctx.every, adj)
        ctx.sim.close()
        f64 = torch.float64
        return (torch.tensor(dE, dtype=f64), torch.tensor(dphi, dtype=f64), g0[:, 0:3].clone(), g0[:, 3:6].clone(),
                None, None, None)


# ------------------------------------------------------------ column collapse

def runout(x: torch.Tensor, axis_xy, p: float = 8.0) -> torch.Tensor:
    """Front runout: the p-norm mean of the particles' horizontal distance
    from the column axis (a smooth stand-in for the largest distance)."""
    d = x[:, :2].double() - torch.as_tensor(axis_xy, dtype=torch.float64, device=x.device)
    r = torch.sqrt((d * d).sum(1) + 1e-12)
    return (r ** p).mean() ** (1.0 / p)


def column_loss(x: torch.Tensor, axis_xy, target) -> torch.Tensor:
    """Squared error of the runout and of the particle-mean position against
    a target (runout, mean) pair."""
    R, m = runout(x, axis_xy), x.double().mean(0)
    return (R - target[0]) ** 2 + ((m - target[1]) ** 2).sum()


def column_target(wl, phi_target: float, nsteps: int):
    """The (runout, mean position) of a forward run at phi_target."""
    from . import mpm as M
    sim = M.Simulation(M.config_from_workload(_with(wl, phi_deg=phi_target), flags=M.DETERMINISTIC), wl.x, wl.v)
    sim.step(nsteps)
    x = torch.tensor(sim.read_particles()["x"], device="cuda")
    sim.close()
    axis = _axis(wl)
    return float(runout(x, axis)), x.double().mean(0)


def _with(wl, **kw):
    import dataclasses
    return dataclasses.replace(wl, **kw)


def _axis(wl):
    return (float(wl.x[:, 0].mean()), float(wl.x[:, 1].mean()))


def column_value_and_grad(wl, phi: float, E: float, target, nsteps: int, every: int):
    """L(phi, E) of the column after nsteps and (dL/dphi, dL/dE)."""
    from . import mpm as M
    x0 = torch.tensor(wl.x, device="cuda")
    v0 = torch.zeros_like(x0)

    def make_sim(E_, phi_, x0_, v0_):
        return M.Simulation(M.config_from_workload(_with(wl, E=E_, phi_deg=phi_), flags=M.DETERMINISTIC), x0_, v0_)

    Et = torch.tensor(E, dtype=torch.float64, requires_grad=True)
    pt = torch.tensor(phi, dtype=torch.float64, requires_grad=True)
    xK, _ = Rollout.apply(Et, pt, x0, v0, make_sim, nsteps, every)
    L = column_loss(xK, _axis(wl), target)
    L.backward()
    return float(L.detach()), float(pt.grad), float(Et.grad)


def calibrate_phi(wl, target, phi0: float, iters: int = 50, lr: float = 0.5, every: int = 20):
    """Adam on phi (degrees) against the target; returns the phi and loss
    history."""
    phi, m, v = phi0, 0.0, 0.0
    b1, b2, eps = 0.9, 0.999, 1e-12
    hist = []
    for t in range(1, iters + 1):
        L, g, _ = column_value_and_grad(wl, phi, wl.E, target, wl.steps, every)
        hist.append((phi, L))
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        phi -= lr * (m / (1 - b1 ** t)) / (((v / (1 - b2 ** t)) ** 0.5) + eps)
    L, _, _ = column_value_and_grad(wl, phi, wl.E, target, wl.steps, every)
    hist.append((phi, L))
    return hist
