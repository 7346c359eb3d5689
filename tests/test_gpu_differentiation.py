"""Differentiation through the library (row a6): the Taylor-deformation loss
and its adjoint, and a multi-step rollout with segment checkpointing, against
reverse-mode differentiation of the FP64 oracle, plus a central-difference
check.  Bar: 1e-4 relative for gradients."""
import numpy as np
import pytest
import torch

from oracle import ibm_oracle as O
from paper_1612_03399_gb300 import _lib
from paper_1612_03399_gb300 import autograd as AG
from paper_1612_03399_gb300 import workloads as W

import helpers as H

pytestmark = pytest.mark.gpu
DEV = "cuda"


def shear_drops(mass=1e-2, dt=2e-3):
    """Three drops (one stretched) in the frozen shear u = y - 1/2, away from
    the y seam; a small node mass so that a few steps deform them.  The
    explicit update needs omega dt < 2 for the stiffest (bending, ~k_b / l^2)
    mode: here omega dt ~ 0.3."""
    rng = np.random.default_rng(2)
    bodies = [W._sphere_body(2, 0.12, np.array([0.3, 0.45, 0.5]), ks=1.0, kb=0.01, mass=mass),
              W._sphere_body(2, 0.1, np.array([0.7, 0.55, 0.35]), rng=rng, stretch=(1.2, 1.0, 0.9),
                             ks=1.5, kb=0.02, mass=mass),
              W._sphere_body(3, 0.09, np.array([0.5, 0.5, 0.8]), ks=0.7, kb=0.005, mass=mass)]
    return W.Workload(name="shear3", bodies=bodies, grid=W.Grid((32, 32, 32)),
                      field={"kind": "shear"}, dt=dt, steps=6)


def test_taylor_deformation_and_adjoint_match_oracle(record_error):
    wl = shear_drops()
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt)
    rel = [r for r in H.rel_positions(wl, W.perturb_positions(wl, 0.05, 4, stretch=0.1))]
    x = H.state_tensor(wl, rel)
    D = ctx.taylor(x).cpu().numpy()
    rng = np.random.default_rng(5)
    gD = rng.standard_normal(len(wl.bodies))
    gx, D2 = ctx.taylor_backward(x, torch.tensor(gD, device=DEV))
    xs = H.split_state(ctx, wl, x)
    ggx = H.split_state(ctx, wl, gx)
    for i, b in enumerate(wl.bodies):
        xt = torch.tensor(xs[i], requires_grad=True)
        Do = O.taylor_deformation(xt, torch.tensor(b.tri, dtype=torch.long), torch.zeros(3, dtype=torch.float64))
        (g,) = torch.autograd.grad(Do * gD[i], xt)
        assert D[i] == pytest.approx(float(Do), rel=1e-9, abs=1e-12)
        record_error(f"gx[{i}]", H.rel_l2(ggx[i], g.numpy()))
        assert H.rel_l2(ggx[i], g.numpy()) <= 1e-6
    assert np.array_equal(D, D2.cpu().numpy())


def oracle_rollout_grads(wl, x0_rel, n_steps, Dstar):
    ob = H.oracle_bodies(wl)
    xs = [torch.tensor(r + b.origin, requires_grad=True) for r, b in zip(x0_rel, wl.bodies)]
    for b in ob:
        b.ks = b.ks.clone().requires_grad_(True)
        b.kb = b.kb.clone().requires_grad_(True)
    prm = H.oracle_params(wl)
    f64 = tuple(t.double() for t in W.sample_field(wl.field, wl.grid, dtype=torch.float64))
    x, v = list(xs), [torch.zeros_like(t) for t in xs]
    for _ in range(n_steps):
        out = O.step(ob, x, v, f64, prm, create_graph=True, with_spread=False)
        x, v = out["x_next"], out["v_next"]
    loss = 0.0
    for i, b in enumerate(ob):
        D = O.taylor_deformation(x[i], b.tri, b.origin)
        loss = loss + (D - Dstar[i]) ** 2
    wrt = xs + [b.ks for b in ob] + [b.kb for b in ob]
    g = torch.autograd.grad(loss, wrt)
    n = len(ob)
    return (float(loss), [t.numpy() for t in g[:n]], np.array([float(t) for t in g[n:2 * n]]),
            np.array([float(t) for t in g[2 * n:]]))


def gpu_rollout_loss(sim, x0, k, n_steps, every, Dstar):
    v0 = torch.zeros_like(x0)
    x, v = AG.rollout(sim, x0, v0, k, n_steps, every)
    D = AG.taylor_deformation(sim, x)
    return ((D - Dstar) ** 2).sum()


def test_rollout_gradients_match_oracle_and_differences(record_error):
    wl = shear_drops()
    n_steps, every = 6, 4                      # two segments: 4 + 2 steps
    rel = H.rel_positions(wl, W.perturb_positions(wl, 0.01, 6))
    sim = AG.Simulation(wl.bodies, wl.grid, wl.field, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    x0 = H.state_tensor(wl, rel).requires_grad_(True)
    x0_rel = [a for a in H.split_state(sim.ctx, wl, x0.detach())]
    Dstar = torch.tensor([0.01, 0.02, 0.005], dtype=torch.float64, device=DEV)
    k = sim.constants().to(DEV).requires_grad_(True)
    loss = gpu_rollout_loss(sim, x0, k, n_steps, every, Dstar)
    loss.backward()
    sim.ctx.check_device_error()
    lo, ogx, ogks, ogkb = oracle_rollout_grads(wl, x0_rel, n_steps, Dstar.cpu().numpy())
    assert float(loss) == pytest.approx(lo, rel=1e-3)
    gk = k.grad.cpu().numpy()
    e_ks = np.linalg.norm(gk[:, 0] - ogks) / np.linalg.norm(ogks)
    e_kb = np.linalg.norm(gk[:, 1] - ogkb) / np.linalg.norm(ogkb)
    record_error("g_ks", e_ks)
    record_error("g_kb", e_kb)
    assert e_ks <= 1e-4 and e_kb <= 1e-4, (gk[:, :2], ogks, ogkb)
    ggx = H.split_state(sim.ctx, wl, x0.grad)
    for i in range(len(wl.bodies)):
        record_error(f"g_x0[{i}]", H.rel_l2(ggx[i], ogx[i]))
        assert H.rel_l2(ggx[i], ogx[i]) <= 1e-4
    # central difference of the GPU loss along k_s -> k_s (1 + eps) for every
    # body.  Float32 positions make D uncertain by ~1e-7, so the loss change
    # must be large: the loss is linear in this direction to 3e-6 over
    # eps = 0.5 (checked in float64 with the oracle), and the bar is loose.
    # The 1e-4 bar against differences is met in float64 by the oracle, whose
    # reverse mode the GPU adjoint matches above.
    eps = 0.5
    vals = []
    for s in (1.0, -1.0):
        kk = k.detach().clone()
        kk[:, 0] *= 1.0 + s * eps
        with torch.no_grad():
            vals.append(float(gpu_rollout_loss(sim, x0.detach(), kk, n_steps, every, Dstar)))
    fd = (vals[0] - vals[1]) / (2 * eps)
    directional = float((gk[:, 0] * k.detach().cpu().numpy()[:, 0]).sum())
    record_error("fd_ks_directional", abs(fd - directional) / abs(directional))
    assert fd == pytest.approx(directional, rel=5e-2)


def test_calibration_lowers_the_loss(record_error):
    """Gradient descent on log k_s, log k_b per drop (calibrate.py) lowers
    sum (D - D*)^2 over a few iterations, targets above the initial D."""
    from paper_1612_03399_gb300.autograd import Simulation
    from paper_1612_03399_gb300.calibrate import calibrate
    wl = shear_drops()
    sim = Simulation(wl.bodies, wl.grid, wl.field, dt=wl.dt)
    x0, v0 = sim.ctx.init_state()
    target = np.array([0.05, 0.08, 0.06])
    _, hist = calibrate(sim, x0, v0, target, n_steps=6, checkpoint_every=3, iters=4, lr=0.3)
    losses = [h["loss"] for h in hist]
    record_error("calibration_loss_ratio", losses[-1] / losses[0])
    assert all(b < a for a, b in zip(losses, losses[1:])), losses
