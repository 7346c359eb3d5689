"""Gradient-descent calibration of per-body elastic constants to target drop
deformations.

The paper tunes ad-hoc elastic constants for drops by comparing simulated
deformations with known ones (Sec. 3.1, Taylor deformation D = (L - B)/(L + B)
in shear).  With the library's adjoint this becomes an optimisation: per
body, log k_s and log k_b (positive by construction) are fitted so that D
after n steps approaches a target D*, loss = sum_b (D_b - D*_b)^2, the
gradient flowing through `rollout` (ibm_step forward, ibm_backward with
segment checkpointing) and `taylor_deformation` (ibm_taylor_backward).

    python -m paper_1612_03399_gb300.calibrate --bodies 256 --steps 50 --iters 5

The explicit step must stay stable for the constants the optimiser visits:
the stiffest (bending) mode has omega ~ sqrt(k_b / (m l^2)) times a geometric
factor, and omega dt must stay well below 2; lowering the node mass makes the
drops deform more within n steps but needs a proportionally smaller dt.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import time

import numpy as np
import torch

from . import workloads as W
from .autograd import Simulation, rollout, taylor_deformation


def calibrate(sim: Simulation, x0, v0, D_target, n_steps: int, checkpoint_every: int = 10,
              iters: int = 10, lr: float = 0.1, callback=None):
    """Fit (k_s, k_b) per body; the other constants stay fixed.  Returns the
    final constants [B, 5] (float64, CPU) and a list of per-iteration records
    (loss, mean |D - D*|, seconds)."""
    base = sim.constants()
    theta = torch.log(base[:, :2]).clone().requires_grad_(True)
    opt = torch.optim.Adam([theta], lr=lr)
    target = torch.as_tensor(D_target, dtype=torch.float64, device=sim.ctx.device)
    history = []
    for it in range(iters):
        torch.cuda.synchronize(sim.ctx.device)
        t0 = time.perf_counter()
        k = torch.cat([theta.exp(), base[:, 2:]], 1)
        xn, _ = rollout(sim, x0, v0, k, n_steps, checkpoint_every)
        D = taylor_deformation(sim, xn)
        loss = ((D - target) ** 2).sum()
        opt.zero_grad()
        loss.backward()
        opt.step()
        torch.cuda.synchronize(sim.ctx.device)
        Dd = D.detach()
        rec = {"iter": it, "loss": float(loss.detach()),
               "mean_abs_dD": float((Dd - target).abs().mean()), "mean_D": float(Dd.mean()),
               "seconds": time.perf_counter() - t0}
        history.append(rec)
        if callback:
            callback(rec)
    k = torch.cat([theta.detach().exp(), base[:, 2:]], 1)
    return k, history


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--bodies", type=int, default=256)
    ap.add_argument("--level", type=int, default=4)
    ap.add_argument("--grid", type=int, default=256)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--checkpoint", type=int, default=10)
    ap.add_argument("--iters", type=int, default=5)
    ap.add_argument("--lr", type=float, default=0.1)
    ap.add_argument("--dt", type=float, default=1e-3)
    ap.add_argument("--mass", type=float, default=1.0)
    ap.add_argument("--mu", type=float, default=1.0)
    args = ap.parse_args(argv)
    wl = W.shear_drops(args.bodies, args.level, args.grid)
    bodies = [dataclasses.replace(b, mass=args.mass) for b in wl.bodies]
    sim = Simulation(bodies, wl.grid, wl.field, dt=args.dt, mu=args.mu)
    x0, v0 = sim.ctx.init_state()
    target = wl.notes["D_target"]
    print(json.dumps({"workload": wl.name, "bodies": len(bodies), "vertices": sim.ctx.V,
                      "steps": args.steps, "checkpoint_every": args.checkpoint}), flush=True)

    def show(rec):
        # one iteration = n forward steps, n recomputed steps and n adjoint steps
        rec["node_steps_per_s_fwd_bwd"] = sim.ctx.V * args.steps / rec["seconds"]
        print(json.dumps(rec), flush=True)

    calibrate(sim, x0, v0, target, args.steps, args.checkpoint, args.iters, args.lr, show)


if __name__ == "__main__":
    main()
