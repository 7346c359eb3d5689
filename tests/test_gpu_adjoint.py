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


def oracle_vjp_spread(wl, ob, xs, vs, fields64, gxn, gvn, gf):
    """Reverse mode of the oracle step including the spread force fields."""
    xs = [x.clone().requires_grad_(True) for x in xs]
    vs = [v.clone().requires_grad_(True) for v in vs]
    for b in ob:
        for k in PARAMS:
            setattr(b, k, getattr(b, k).clone().requires_grad_(True))
    out = O.step(ob, xs, vs, fields64, H.oracle_params(wl), create_graph=True, with_spread=True)
    J = sum((out["x_next"][i] * gxn[i]).sum() + (out["v_next"][i] * gvn[i]).sum()
            for i in range(len(ob)))
    J = J + (out["f"] * gf).sum()
    wrt = xs + vs + [getattr(b, k) for b in ob for k in PARAMS]
    grads = torch.autograd.grad(J, wrt, allow_unused=True)
    n = len(ob)
    gx = [g.detach().numpy() for g in grads[:n]]
    gv = [g.detach().numpy() for g in grads[n:2 * n]]
    gp = np.array([[0.0 if g is None else float(g) for g in grads[2 * n + 5 * i:2 * n + 5 * i + 5]]
                   for i in range(n)])
    return gx, gv, gp


def test_backward_with_spread_cotangent_matches_oracle(record_error):
    """ibm_backward with cotangents of the spread force fields (Eq. mls_cl;
    spreading transposed is interpolation weighted by c_l) and nonzero vertex
    velocities, against the oracle's reverse mode through the spread."""
    wl = mixed_workload()
    ob = H.oracle_bodies(wl)
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    rel = tie_free_state(wl, 30, scale=0.05, stretch=0.05)
    x = H.state_tensor(wl, rel)
    xs = H.to_abs(wl, H.split_state(ctx, wl, x))
    rng = np.random.default_rng(31)
    v = torch.tensor(rng.uniform(-0.3, 0.3, (3, ctx.V)), dtype=torch.float32, device=DEV)
    gxn = torch.tensor(rng.standard_normal((3, ctx.V)), dtype=torch.float32, device=DEV)
    gvn = torch.tensor(rng.standard_normal((3, ctx.V)), dtype=torch.float32, device=DEV)
    nx, ny, nz = wl.grid.n
    gf = torch.tensor(rng.standard_normal((3, nz, ny, nx)), dtype=torch.float32, device=DEV)
    fields = H.fields_for(wl, DEV)
    gx, gv, gp = ctx.backward(x, fields, gxn, gvn, v=v, gf=(gf[0], gf[1], gf[2]))
    ctx.check_device_error()
    vs = [torch.tensor(a) for a in H.split_state(ctx, wl, v)]
    gxn_b = [torch.tensor(a) for a in H.split_state(ctx, wl, gxn)]
    gvn_b = [torch.tensor(a) for a in H.split_state(ctx, wl, gvn)]
    ogx, ogv, ogp = oracle_vjp_spread(wl, ob, xs, vs, tuple(f.double().cpu() for f in fields),
                                      gxn_b, gvn_b, gf.double().cpu())
    ggx = H.split_state(ctx, wl, gx)
    ggv = H.split_state(ctx, wl, gv)
    gp = gp.cpu().numpy()
    for i, b in enumerate(wl.bodies):
        d_g = ggx[i] - gxn_b[i].numpy()
        d_o = ogx[i] - gxn_b[i].numpy()
        record_error(f"gx[{i}]", H.rel_l2(d_g, d_o))
        assert H.rel_l2(d_g, d_o) <= 1e-4, (i, H.rel_l2(d_g, d_o))
        cl = b.clamped[:, None] if b.clamped is not None else np.zeros((len(b.rest), 1), bool)
        base = np.where(cl, 0.0, gvn_b[i].numpy() + wl.dt * gxn_b[i].numpy())
        e_v = H.rel_l2(ggv[i] - base, ogv[i] - base)
        record_error(f"gv[{i}]", e_v)
        assert e_v <= 1e-4, (i, e_v)
        for k, name in enumerate(PARAMS):
            if b.closed is False and name == "kv":
                continue
            err = abs(gp[i, k] - ogp[i, k]) / max(abs(ogp[i, k]), 1e-30)
            assert err <= 1e-4, (i, name, gp[i, k], ogp[i, k])


def affine_mac(wl, A, b, device):
    """Fields q_i = A[i] . x + b[i] sampled at the MAC nodes of component i
    ([3, nz, ny, nx] float32)."""
    nx, ny, nz = wl.grid.n
    h = wl.grid.h
    out = []
    offs = ((0.0, 0.5, 0.5), (0.5, 0.0, 0.5), (0.5, 0.5, 0.0))
    for i in range(3):
        zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        X = ((xx + offs[i][0]) * h[0], (yy + offs[i][1]) * h[1], (zz + offs[i][2]) * h[2])
        out.append(A[i][0] * X[0] + A[i][1] * X[1] + A[i][2] * X[2] + b[i])
    return torch.tensor(np.stack(out), dtype=torch.float32, device=device)


def test_backward_dot_product_with_step_differences(record_error):
    """Dot-product test on the GPU alone: for the step map S: (x, v) ->
    (x', v', f) and a cotangent w = (w_x, w_v, w_f), <w, (S(z + d) - S(z -
    d))/2> = <d, S^T w> with S^T w from ibm_backward (field cotangents
    included).  The flow and w_f are affine fields, which MLS reproduces
    exactly with any stencil, so <w, S(z)> is smooth in z whatever nodes the
    markers pick; a transposed or misplaced term of the adjoint breaks the
    identity by O(1)."""
    wl = mixed_workload()
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    h = float(min(wl.grid.h))
    rng = np.random.default_rng(41)
    rel = deformed_state(wl, 40, scale=0.03, stretch=0.03)
    x = H.state_tensor(wl, rel)
    v = torch.tensor(rng.uniform(-0.3, 0.3, (3, ctx.V)), dtype=torch.float32, device=DEV)
    dx = torch.tensor(rng.uniform(-1, 1, (3, ctx.V)) * 2e-2 * h, dtype=torch.float32, device=DEV)
    dv = torch.tensor(rng.uniform(-1, 1, (3, ctx.V)) * 1e-2, dtype=torch.float32, device=DEV)
    for i, b in enumerate(wl.bodies):   # clamped nodes stay fixed in position
        if b.clamped is not None:
            o = int(ctx.v_off[i])
            dx[:, o:o + len(b.rest)][:, torch.tensor(b.clamped, device=DEV)] = 0.0
    u = affine_mac(wl, rng.uniform(-1, 1, (3, 3)), rng.uniform(-0.5, 0.5, 3), DEV)
    fields = (u[0].contiguous(), u[1].contiguous(), u[2].contiguous())
    wf = affine_mac(wl, rng.uniform(-1, 1, (3, 3)), rng.uniform(-0.5, 0.5, 3), DEV)
    wx = torch.tensor(rng.standard_normal((3, ctx.V)), dtype=torch.float32, device=DEV)
    wv = torch.tensor(rng.standard_normal((3, ctx.V)), dtype=torch.float32, device=DEV)
    nx, ny, nz = wl.grid.n

    def S(xx, vv):
        f = tuple(torch.zeros((nz, ny, nx), dtype=torch.float32, device=DEV) for _ in range(3))
        x1, v1 = torch.empty_like(xx), torch.empty_like(vv)
        ctx.step(xx, vv, fields, x1, v1, f, clear=False)
        ctx.check_device_error()
        return x1.double(), v1.double(), torch.stack(f).double()

    xp, vp, fp = S(x + dx, v + dv)
    xm, vm, fm = S(x - dx, v - dv)
    lhs = 0.5 * float((wx.double() * (xp - xm)).sum() + (wv.double() * (vp - vm)).sum()
                      + (wf.double() * (fp - fm)).sum())
    gx, gv, _ = ctx.backward(x, fields, wx, wv, v=v, gf=(wf[0].contiguous(), wf[1].contiguous(),
                                                        wf[2].contiguous()))
    rhs = float((gx.double() * dx.double()).sum() + (gv.double() * dv.double()).sum())
    err = abs(lhs - rhs) / abs(rhs)
    record_error("dot", err)
    assert err <= 1e-3, (lhs, rhs, err)
