"""Strong coupling on the GPU (ibm_step_pc): Hamming's predictor-corrector
with the Runge-Kutta start against the FP64 oracle over a trajectory,
through the C ABI.

Bar: positions (body frame, relative to the body size) and velocity changes
(beyond half an ulp of float32 storage per step taken) within 1e-5 after
every step; clamped nodes stay put; ibm_pc_reset restarts
the same trajectory bit for bit."""
import numpy as np
import pytest
import torch

from oracle import ibm_oracle as O
from paper_1612_03399_gb300 import _lib

import helpers as H
from test_gpu_parity import mixed_workload, tie_free_state

pytestmark = pytest.mark.gpu
DEV = "cuda"
STEPS = 8


def run_gpu(ctx, x, v, fields, wl, steps=STEPS):
    n = wl.grid.n
    f = tuple(torch.zeros((n[2], n[1], n[0]), dtype=torch.float32, device=DEV) for _ in range(3))
    out = []
    for _ in range(steps):
        x1, v1 = torch.empty_like(x), torch.empty_like(v)
        ctx.step_pc(x, v, fields, x1, v1, f)
        out.append((x1, v1))
        x, v = x1, v1
    ctx.check_device_error()
    return out


def test_trajectory_matches_oracle(record_error):
    wl = mixed_workload()
    ob = H.oracle_bodies(wl)
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    rel = tie_free_state(wl, 30, scale=0.03, stretch=0.03)
    x = H.state_tensor(wl, rel)
    rng = np.random.default_rng(2)
    v = torch.tensor(rng.uniform(-0.2, 0.2, (3, ctx.V)), dtype=torch.float32, device=DEV)
    # clamped nodes start at rest (they stay so)
    cl = np.concatenate([b.clamped if b.clamped is not None else np.zeros(len(b.rest), bool)
                         for b in wl.bodies])
    v[:, torch.tensor(cl, device=DEV)] = 0.0
    fields = H.fields_for(wl, DEV)
    traj = run_gpu(ctx, x, v, fields, wl)
    xs = H.to_abs(wl, H.split_state(ctx, wl, x))
    vs = [torch.tensor(t) for t in H.split_state(ctx, wl, v)]
    ref = O.hamming_rollout(ob, xs, vs, tuple(t.double().cpu() for t in fields),
                            H.oracle_params(wl), STEPS)
    x0 = H.split_state(ctx, wl, x)
    for k in range(STEPS):
        xg = H.split_state(ctx, wl, traj[k][0])
        vg = H.split_state(ctx, wl, traj[k][1])
        for i, b in enumerate(wl.bodies):
            size = float(np.linalg.norm(b.rest - b.origin, axis=1).max())
            xo = ref[k][0][i].numpy() - b.origin
            ex = np.linalg.norm(xg[i] - xo) / (size * np.sqrt(len(xo)))
            # velocity change beyond the float32 storage of the velocity: half an
            # ulp per stored step, k + 1 of them after step k (each step's
            # output is the next step's input)
            vo = ref[k][1][i].numpy()
            dvo = vo - vs[i].numpy()
            store = (k + 1) * np.linalg.norm(
                0.5 * np.spacing(np.abs(vo).astype(np.float32)).astype(np.float64))
            ev = max(0.0, np.linalg.norm((vg[i] - vs[i].numpy()) - dvo) - store) / np.linalg.norm(dvo)
            record_error(f"x[{k}][{i}]", ex)
            record_error(f"dv[{k}][{i}]", ev)
            assert ex <= 1e-5, (k, i, ex)
            assert ev <= 1e-5, (k, i, ev)
            if b.clamped is not None:
                assert np.array_equal(xg[i][b.clamped], x0[i][b.clamped])
                assert not vg[i][b.clamped].any()


def test_reset_restarts_the_trajectory_bitwise():
    wl = mixed_workload()
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    x, v = ctx.init_state()
    fields = H.fields_for(wl, DEV)
    a = run_gpu(ctx, x, v, fields, wl, 6)
    ctx.pc_reset()
    b = run_gpu(ctx, x, v, fields, wl, 6)
    for (xa, va), (xb, vb) in zip(a, b):
        assert torch.equal(xa, xb) and torch.equal(va, vb)
