"""The hand-written adjoint of one step (ibm_backward) against reverse-mode
differentiation of the FP64 oracle step, through the C ABI.

Bar: the non-trivial part of the position cotangent (gx - gx', which carries
the force Hessian and the traction adjoint) and the constants' cotangents
within 1e-4 relative L2 per body; gv exact up to float32 rounding."""
import numpy as np
import pytest
import torch

from oracle import ibm_oracle as O
from paper_1612_03399_gb300 import _lib
from paper_1612_03399_gb300 import workloads as W

import helpers as H
from test_gpu_parity import deformed_state, mixed_workload, tie_free_state

pytestmark = pytest.mark.gpu
DEV = "cuda"
PARAMS = ["ks", "kb", "ka", "kA", "kv"]


def oracle_vjp(wl, ob, xs, vs, fields64, gxn, gvn, forward_euler=False):
    xs = [x.clone().requires_grad_(True) for x in xs]
    vs = [v.clone().requires_grad_(True) for v in vs]
    for b in ob:
        for k in PARAMS:
            setattr(b, k, getattr(b, k).clone().requires_grad_(True))
    out = O.step(ob, xs, vs, fields64, H.oracle_params(wl, forward_euler=forward_euler),
                 create_graph=True, with_spread=False)
    J = sum((out["x_next"][i] * gxn[i]).sum() + (out["v_next"][i] * gvn[i]).sum()
            for i in range(len(ob)))
    wrt = xs + vs + [getattr(b, k) for b in ob for k in PARAMS]
    grads = torch.autograd.grad(J, wrt, allow_unused=True)
    n = len(ob)
    gx = [g.detach().numpy() for g in grads[:n]]
    gv = [g.detach().numpy() for g in grads[n:2 * n]]
    gp = np.array([[0.0 if g is None else float(g) for g in grads[2 * n + 5 * i:2 * n + 5 * i + 5]]
                   for i in range(n)])
    return gx, gv, gp


@pytest.mark.parametrize("forward_euler", [False, True])
def test_backward_matches_oracle_reverse_mode(forward_euler, record_error):
    wl = mixed_workload()
    ob = H.oracle_bodies(wl)
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha,
                       forward_euler=forward_euler)
    rel = tie_free_state(wl, 20, scale=0.05, stretch=0.05)
    x = H.state_tensor(wl, rel)
    xs = H.to_abs(wl, H.split_state(ctx, wl, x))
    rng = np.random.default_rng(9)
    gxn_np = rng.standard_normal((3, ctx.V))
    gvn_np = rng.standard_normal((3, ctx.V))
    gxn = torch.tensor(gxn_np, dtype=torch.float32, device=DEV)
    gvn = torch.tensor(gvn_np, dtype=torch.float32, device=DEV)
    fields = H.fields_for(wl, DEV)
    gx, gv, gp = ctx.backward(x, fields, gxn, gvn)
    ctx.check_device_error()
    vs = [torch.zeros_like(t) for t in xs]
    gxn_b = [torch.tensor(a) for a in H.split_state(ctx, wl, gxn)]
    gvn_b = [torch.tensor(a) for a in H.split_state(ctx, wl, gvn)]
    ogx, ogv, ogp = oracle_vjp(wl, ob, xs, vs, tuple(f.double().cpu() for f in fields), gxn_b,
                               gvn_b, forward_euler)
    ggx = H.split_state(ctx, wl, gx)
    ggv = H.split_state(ctx, wl, gv)
    gp = gp.cpu().numpy()
    for i, b in enumerate(wl.bodies):
        d_g = ggx[i] - gxn_b[i].numpy()
        d_o = ogx[i] - gxn_b[i].numpy()
        record_error(f"gx[{i}]", H.rel_l2(d_g, d_o))
        assert H.rel_l2(d_g, d_o) <= 1e-4, (i, H.rel_l2(d_g, d_o))
        assert H.rel_l2(ggv[i], ogv[i]) <= 1e-6, i
        for k, name in enumerate(PARAMS):
            if b.closed is False and name == "kv":
                assert gp[i, k] == 0.0
                continue
            err = abs(gp[i, k] - ogp[i, k]) / max(abs(ogp[i, k]), 1e-30)
            record_error(f"g{name}[{i}]", err)
            assert err <= 1e-4, (i, name, gp[i, k], ogp[i, k])


def test_backward_is_deterministic():
    wl = mixed_workload()
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt)
    x = H.state_tensor(wl, deformed_state(wl, 3))
    rng = np.random.default_rng(1)
    gxn = torch.tensor(rng.standard_normal((3, ctx.V)), dtype=torch.float32, device=DEV)
    gvn = torch.tensor(rng.standard_normal((3, ctx.V)), dtype=torch.float32, device=DEV)
    fields = H.fields_for(wl, DEV)
    a = ctx.backward(x, fields, gxn, gvn)
    b = ctx.backward(x, fields, gxn, gvn)
    for p, q in zip(a, b):
        assert torch.equal(p, q)
