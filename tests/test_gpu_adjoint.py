"""The hand-written adjoint of the explicit step (deterministic mode) against
FP64 central differences of the oracle: one step for every input family (x,
v, C, F, Young's modulus E and, for Drucker-Prager, the friction angle phi),
and checkpointed rollouts through the torch.autograd.Function."""
import numpy as np
import pytest

from paper_2605_28525_b300 import mpm, workloads as W
from tests.helpers import oracle_for, small_blob

pytestmark = pytest.mark.gpu


def _blob(floor=False, dp=False, fscale=0.03):
    wl, Cm, F = small_blob(n=2000, seed=21, E=1e5, vscale=0.5, cscale=2.0, fscale=fscale, dt=2e-4,
                           material=W.DRUCKER_PRAGER if dp else W.NEOHOOKEAN)
    if dp:
        # per-particle friction angles (degrees)
        wl.phi = np.random.default_rng(4).uniform(25.0, 35.0, wl.n).astype(np.float32)
    if floor:
        # a Coulomb floor under the blob's lower cells
        wl.floor_kind, wl.floor_z, wl.floor_mu = W.FLOOR_COULOMB, 12 * wl.dx, 0.3
    return wl, Cm.reshape(-1, 9), F.reshape(-1, 9)


def _oracle(wl, E):
    import dataclasses
    return oracle_for(dataclasses.replace(wl, E=E))


def _L(out, wts):
    x, v, Cm, F = out
    a, b, ca, fa = wts
    return float((x * a).sum() + (v * b).sum() + (Cm.reshape(-1, 9) * ca).sum() + (F.reshape(-1, 9) * fa).sum())


def _pick(x, h, rng, k):
    """Particles whose cell offsets stay clear of the cell faces (the
    stencil must not change under the finite differences)."""
    d = x / h - np.floor(x / h - 0.5)
    ok = np.all((d > 0.52) & (d < 1.48), axis=1)
    return rng.choice(np.flatnonzero(ok), k, replace=False)


# fscale 0.03 puts most particles' ||F F^T - I|| above 1/16 (the return map and
# Hencky stress adjoints through the FP64 SVD), 0.005 below it (their series forms)
@pytest.mark.parametrize("floor,dp,fscale", [(False, False, 0.03), (True, False, 0.03), (False, True, 0.03),
                                             (True, True, 0.03), (False, True, 0.005), (True, True, 0.005)])
def test_one_step_adjoint_matches_fp64_differences(oracle_mod, floor, dp, fscale):
    import torch
    wl, Cm, F = _blob(floor, dp, fscale)
    n = wl.n
    rng = np.random.default_rng(5)
    wts = (rng.standard_normal((n, 3)), rng.standard_normal((n, 3)), rng.standard_normal((n, 9)) * 1e-2,
           rng.standard_normal((n, 9)))
    sim = mpm.Simulation(mpm.config_from_workload(wl, flags=mpm.DETERMINISTIC), wl.x, wl.v, Cm, F, phi=wl.phi)
    adj_next = torch.tensor(np.concatenate(wts, axis=1), dtype=torch.float32, device="cuda")
    adj_cur = torch.empty_like(adj_next)
    dE, dphi = sim.adjoint_step(adj_next, adj_cur)
    g = adj_cur.cpu().numpy().astype(np.float64)

    x0, v0, C0, F0 = (a.astype(np.float64) for a in (wl.x, wl.v, Cm, F))
    phi0 = None if wl.phi is None else wl.phi.astype(np.float64)
    o = oracle_for(wl)

    def L_of(x=x0, v=v0, C_=C0, F_=F0, orc=o, phi=phi0):
        return _L(orc.run(x, v, C_, F_, phi, nsteps=1), wts)

    # E
    dEr = 1e-5 * wl.E
    fd = (L_of(orc=_oracle(wl, wl.E + dEr)) - L_of(orc=_oracle(wl, wl.E - dEr))) / (2 * dEr)
    assert fd != 0.0
    assert abs(dE - fd) <= 1e-3 * abs(fd), (dE, fd)
    if dp:   # phi of every particle moved together
        fdp = (L_of(phi=phi0 + 1e-4) - L_of(phi=phi0 - 1e-4)) / 2e-4
        assert fdp != 0.0
        assert abs(dphi - fdp) <= 1e-3 * abs(fdp), (dphi, fdp)
    # x, v, C, F of sampled particles
    ps = _pick(wl.x, wl.dx, rng, 6)
    fams = {"x": (x0, 0, 3, 1e-5 * wl.dx), "v": (v0, 3, 3, 1e-5), "C": (C0, 6, 9, 1e-4), "F": (F0, 15, 9, 1e-6)}
    for name, (arr, off, width, eps) in fams.items():
        got, want = [], []
        for p in ps:
            for k in range(width):
                a1, a2 = arr.copy(), arr.copy()
                a1[p, k] += eps
                a2[p, k] -= eps
                kw1, kw2 = {"x": {}, "v": {}, "C": {}, "F": {}}[name], {}
                args1 = dict(x=x0, v=v0, C_=C0, F_=F0)
                args2 = dict(args1)
                key = {"x": "x", "v": "v", "C": "C_", "F": "F_"}[name]
                args1[key], args2[key] = a1, a2
                want.append((L_of(**args1) - L_of(**args2)) / (2 * eps))
                got.append(g[p, off + k])
        got, want = np.array(got), np.array(want)
        assert np.abs(want).max() > 0
        assert np.abs(got - want).max() <= 1e-3 * np.abs(want).max(), (name, got, want)


def test_checkpointed_rollout_gradient(oracle_mod):
    import torch
    from paper_2605_28525_b300 import adjoint
    wl, Cm, F = _blob()
    n, K = wl.n, 24
    rng = np.random.default_rng(8)
    cx, cv = rng.standard_normal((n, 3)), rng.standard_normal((n, 3))
    C_d = torch.tensor(Cm, device="cuda")
    F_d = torch.tensor(F, device="cuda")

    def make_sim(E, phi, x0, v0):
        import dataclasses
        cfg = mpm.config_from_workload(dataclasses.replace(wl, E=E), flags=mpm.DETERMINISTIC)
        return mpm.Simulation(cfg, x0, v0, C_d, F_d)

    grads = []
    for every in (7, K):
        E = torch.tensor(wl.E, dtype=torch.float64, requires_grad=True)
        phi = torch.tensor(30.0, dtype=torch.float64)
        x0 = torch.tensor(wl.x, device="cuda", requires_grad=True)
        v0 = torch.tensor(wl.v, device="cuda", requires_grad=True)
        xK, vK = adjoint.Rollout.apply(E, phi, x0, v0, make_sim, K, every)
        loss = (xK.double() * torch.tensor(cx, device="cuda")).sum() + \
               (vK.double() * torch.tensor(cv, device="cuda")).sum()
        loss.backward()
        grads.append((float(E.grad), v0.grad.cpu().numpy().astype(np.float64), loss.item()))
    # checkpointing changes nothing but the float-atomic order of the node adjoints
    assert abs(grads[0][0] - grads[1][0]) <= 1e-5 * abs(grads[1][0])
    assert np.allclose(grads[0][1], grads[1][1], rtol=1e-4, atol=1e-6 * np.abs(grads[1][1]).max())

    x0d, v0d, C0d, F0d = (a.astype(np.float64) for a in (wl.x, wl.v, Cm, F))

    def L_of(E=wl.E, v=v0d):
        x, vv, _, _ = _oracle(wl, E).run(x0d, v, C0d, F0d, nsteps=K)
        return float((x * cx).sum() + (vv * cv).sum())

    dEr = 1e-5 * wl.E
    fd = (L_of(E=wl.E + dEr) - L_of(E=wl.E - dEr)) / (2 * dEr)
    assert abs(grads[0][0] - fd) <= 1e-3 * abs(fd), (grads[0][0], fd)
    got, want = [], []
    for p in _pick(wl.x, wl.dx, rng, 4):
        for k in range(3):
            a1, a2 = v0d.copy(), v0d.copy()
            a1[p, k] += 1e-5
            a2[p, k] -= 1e-5
            want.append((L_of(v=a1) - L_of(v=a2)) / 2e-5)
            got.append(grads[0][1][p, k])
    got, want = np.array(got), np.array(want)
    assert np.abs(got - want).max() <= 1e-3 * np.abs(want).max(), (got, want)


def test_dp_rollout_gradient_phi_and_E(oracle_mod):
    """20 Drucker-Prager steps of a blob pressed onto a Coulomb floor,
    checkpoints every 6: dL/dphi and dL/dE of its mean position (weighted
    per axis) against FP64 differences."""
    import torch
    from paper_2605_28525_b300 import adjoint
    wl, Cm, F = _blob(floor=True, dp=True)
    n, K = wl.n, 20
    c = np.tile(np.array([[0.2, 0.1, 1.0]]), (n, 1)) / n
    sim = mpm.Simulation(mpm.config_from_workload(wl, flags=mpm.DETERMINISTIC), wl.x, wl.v, Cm, F, phi=wl.phi)
    ckpts = adjoint.rollout(sim, K, 6)
    adj = torch.zeros(n, 24, dtype=torch.float32, device="cuda")
    adj[:, 0:3] = torch.tensor(c, dtype=torch.float32, device="cuda")
    _, dE, dphi = adjoint.gradient(sim, ckpts, K, 6, adj)
    x0, v0, C0, F0 = (a.astype(np.float64) for a in (wl.x, wl.v, Cm, F))
    phi0 = wl.phi.astype(np.float64)

    def L_of(E=wl.E, phi=phi0):
        x, _, _, _ = _oracle(wl, E).run(x0, v0, C0, F0, phi, nsteps=K)
        return float((x * c).sum())

    fdp = (L_of(phi=phi0 + 1e-5) - L_of(phi=phi0 - 1e-5)) / 2e-5
    fdE = (L_of(E=wl.E * (1 + 1e-6)) - L_of(E=wl.E * (1 - 1e-6))) / (2e-6 * wl.E)
    assert fdp != 0.0 and fdE != 0.0
    assert abs(dphi - fdp) <= 1e-3 * abs(fdp), (dphi, fdp)
    assert abs(dE - fdE) <= 1e-3 * abs(fdE), (dE, fdE)


def test_adjoint_refuses_unsupported_contexts(oracle_mod):
    import torch
    wl, Cm, F = _blob()
    adj = torch.zeros(wl.n, 24, device="cuda")
    for flags, mat in [(0, W.NEOHOOKEAN), (0, W.DRUCKER_PRAGER)]:
        wl.material = mat
        sim = mpm.Simulation(mpm.config_from_workload(wl, flags=flags), wl.x, wl.v, Cm, F)
        with pytest.raises(mpm.MpmError) as e:
            sim.adjoint_step(adj, torch.empty_like(adj))
        assert e.value.status == mpm.ERR_INVALID_ARG


def test_column_functional_gradient_matches_fp64(oracle_mod):
    """The differentiable column's geometry (an 8^3-cell cube), squeezed by
    an initial velocity field towards its centre so that 50 steps see both
    the elastic and the plastic response, without a floor (a body at rest
    on a Coulomb floor keeps nodes on the kinks of the friction law, where
    central differences of a 50-step trajectory are not smooth; the floor's
    adjoint is checked step by step above): the gradient of the front runout
    plus a weighted mean position with respect to phi and E, through the
    checkpointed autograd.Function, against FP64 central differences of the
    same functional on the oracle's trajectories."""
    import dataclasses
    import torch
    from paper_2605_28525_b300 import adjoint
    wl = W.diff_column(cells=8, steps=50, box=(32, 32, 24))
    wl = dataclasses.replace(wl, floor_kind=W.FLOOR_NONE, gravity=(0.0, 0.0, 0.0))
    c = wl.x.astype(np.float64).mean(0)
    v0n = (-4.0 * (wl.x - c) * np.array([1.0, 1.0, 0.5])).astype(np.float32)
    axis = adjoint._axis(wl)
    wts = torch.tensor([0.3, 0.2, 1.0], dtype=torch.float64)

    def J(x):
        return adjoint.runout(x, axis) + (x.double().mean(0) * wts.to(x.device)).sum()

    def make_sim(E_, phi_, x0_, v0_):
        return mpm.Simulation(mpm.config_from_workload(dataclasses.replace(wl, E=E_, phi_deg=phi_),
                                                       flags=mpm.DETERMINISTIC), x0_, v0_)

    Et = torch.tensor(wl.E, dtype=torch.float64, requires_grad=True)
    pt = torch.tensor(30.0, dtype=torch.float64, requires_grad=True)
    x0 = torch.tensor(wl.x, device="cuda")
    xK, _ = adjoint.Rollout.apply(Et, pt, x0, torch.tensor(v0n, device="cuda"), make_sim, wl.steps, 16)
    J(xK).backward()

    def J_of(phi=30.0, E=wl.E):
        o = oracle_for(dataclasses.replace(wl, E=E, phi_deg=phi))
        x, _, _, _ = o.run(wl.x.astype(np.float64), v0n.astype(np.float64), nsteps=wl.steps)
        return float(J(torch.tensor(x)))

    fdp = (J_of(phi=30.0 + 1e-5) - J_of(phi=30.0 - 1e-5)) / 2e-5
    fdE = (J_of(E=wl.E * (1 + 1e-6)) - J_of(E=wl.E * (1 - 1e-6))) / (2e-6 * wl.E)
    assert fdp != 0.0 and fdE != 0.0
    assert abs(float(pt.grad) - fdp) <= 1e-3 * abs(fdp), (float(pt.grad), fdp)
    assert abs(float(Et.grad) - fdE) <= 1e-3 * abs(fdE), (float(Et.grad), fdE)


def _golden_diff_column():
    import json
    import os
    return json.load(open(os.path.join(os.path.dirname(__file__), "golden", "diff_column_fd.json")))


def test_diff_column_gradients_at_full_configuration(oracle_mod):
    """The differentiable column exactly as configured: 262,144 particles,
    Drucker-Prager phi = 30 deg, E = 5e6 Pa, 400 steps with gravity on the
    Coulomb floor, checkpoints every 20 steps.  The loss (squared error of
    the runout and mean position against the phi = 34 deg run) and its
    gradient through the checkpointed adjoint, against FP64 central
    differences of the oracle's trajectories (tests/golden/diff_column_fd.json,
    written by make_diff_column_fd.py beside it; the target run is the
    oracle's too).  The stored step-size study (three step sizes per
    parameter agreeing to 2e-5) shows the loss is smooth at this point.
    Also the gradient of the runout plus a weighted mean position, a
    functional of the trajectory alone (no target residual)."""
    import torch
    from paper_2605_28525_b300 import adjoint
    g = _golden_diff_column()
    wl = W.diff_column()
    cfg = g["config"]
    assert (wl.n, wl.steps, wl.phi_deg, wl.E) == (cfg["particles"], cfg["steps"], cfg["phi_deg"], cfg["E"])
    assert tuple(cfg["axis"]) == adjoint._axis(wl)
    fdp = g["dL_dphi_per_deg"]["0.001"]
    fdE = g["dL_dE"]["0.0001"]
    # the step-size study: the central differences agree across step sizes
    assert max(abs(v - fdp) for v in g["dL_dphi_per_deg"].values()) <= 1e-4 * abs(fdp)
    assert max(abs(v - fdE) for v in g["dL_dE"].values()) <= 1e-4 * abs(fdE)
    target = (g["target"]["runout"], torch.tensor(g["target"]["mean"], dtype=torch.float64, device="cuda"))
    L, dphi, dE = adjoint.column_value_and_grad(wl, wl.phi_deg, wl.E, target, wl.steps, 20)
    assert abs(L - g["loss"]) <= 1e-2 * g["loss"], (L, g["loss"])
    assert abs(dphi - fdp) <= 1e-3 * abs(fdp), (dphi, fdp)
    assert abs(dE - fdE) <= 1e-3 * abs(fdE), (dE, fdE)

    # J = R + w . mean(x): the trajectory's own functional, from the stored runs
    w = np.array([0.3, 0.2, 1.0])

    def J_run(phi, E):
        r = [r for r in g["runs"] if abs(r["phi_deg"] - phi) < 1e-9 and abs(r["E"] - E) < 1e-6 * E]
        assert len(r) == 1, (phi, E)
        return r[0]["runout"] + float(np.dot(w, r[0]["mean"]))

    hp, he = 1e-3, 1e-4
    fJp = (J_run(wl.phi_deg + hp, wl.E) - J_run(wl.phi_deg - hp, wl.E)) / (2 * hp)
    fJE = (J_run(wl.phi_deg, wl.E * (1 + he)) - J_run(wl.phi_deg, wl.E * (1 - he))) / (2 * he * wl.E)
    axis = adjoint._axis(wl)
    wt = torch.tensor(w, dtype=torch.float64, device="cuda")

    def make_sim(E_, phi_, x0_, v0_):
        import dataclasses
        return mpm.Simulation(mpm.config_from_workload(dataclasses.replace(wl, E=E_, phi_deg=phi_),
                                                       flags=mpm.DETERMINISTIC), x0_, v0_)

    Et = torch.tensor(wl.E, dtype=torch.float64, requires_grad=True)
    pt = torch.tensor(wl.phi_deg, dtype=torch.float64, requires_grad=True)
    x0 = torch.tensor(wl.x, device="cuda")
    xK, _ = adjoint.Rollout.apply(Et, pt, x0, torch.zeros_like(x0), make_sim, wl.steps, 20)
    (adjoint.runout(xK, axis) + (xK.double().mean(0) * wt).sum()).backward()
    assert abs(float(pt.grad) - fJp) <= 1e-3 * abs(fJp), (float(pt.grad), fJp)
    assert abs(float(Et.grad) - fJE) <= 1e-3 * abs(fJE), (float(Et.grad), fJE)
