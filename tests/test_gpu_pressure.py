"""Probe pressure with the marker-acceleration correction (Sec. 2.2) on the
GPU, through the C ABI: traction, step and adjoint against the FP64 oracle,
and the buoyancy closed form on the GPU alone.

Bars as for the viscous traction: relative L2 <= 1e-5 (traction, velocity
increment beyond half an ulp of the stored float32 velocity), adjoint
<= 1e-4; markers within 2e-5 cells of a nearest-node switch are left out."""
import dataclasses

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


def pressure_inputs(wl, ctx, seed):
    rng = np.random.default_rng(seed)
    spec = W.pressure_modes(12, 3, 20.0, rng)
    p = W.sample_pressure(spec, wl.grid, device=DEV, dtype=torch.float32)
    p64 = W.sample_pressure(spec, wl.grid, dtype=torch.float64)
    a = torch.tensor(rng.uniform(-20.0, 20.0, (3, ctx.V)), dtype=torch.float32, device=DEV)
    a_b = [torch.tensor(t) for t in H.split_state(ctx, wl, a)]
    return p, p64, a, a_b


def test_pressure_traction_parity(record_error):
    wl = mixed_workload()
    ob = H.oracle_bodies(wl)
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    x = H.state_tensor(wl, deformed_state(wl, 3, scale=0.02, stretch=0.02))
    v = torch.zeros((3, ctx.V), dtype=torch.float32, device=DEV)
    fields = H.fields_for(wl, DEV)
    p, p64, a, a_b = pressure_inputs(wl, ctx, 11)
    _, _, Fe = ctx.interpolate(x, v, fields, U=False, F_marker=False, F_ext=True, p=p, accel=a)
    _, _, Fe0 = ctx.interpolate(x, v, fields, U=False, F_marker=False, F_ext=True)
    ctx.check_device_error()
    xs = H.to_abs(wl, H.split_state(ctx, wl, x))
    vs = [torch.zeros_like(t) for t in xs]
    f64 = tuple(f.double().cpu() for f in fields)
    out = O.step(ob, xs, vs, f64, H.oracle_params(wl), with_spread=False, pressure=p64, accels=a_b)
    keep = H.tie_mask(wl, xs)
    assert keep.mean() > 0.99
    gg = Fe.double().cpu().numpy().T[keep]
    oo = out["F_ext_face"].numpy()[keep]
    e = H.rel_l2(gg, oo)
    record_error("F_ext_face", e)
    assert e <= 1e-5
    # the pressure part is a substantial share of the load
    assert np.linalg.norm(gg - Fe0.double().cpu().numpy().T[keep]) > 0.3 * np.linalg.norm(oo)


def test_pressure_step_parity(record_error):
    wl = mixed_workload()
    ob = H.oracle_bodies(wl)
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    rel = tie_free_state(wl, 21, scale=0.03, stretch=0.03)
    x = H.state_tensor(wl, rel)
    rng = np.random.default_rng(5)
    v = torch.tensor(rng.uniform(-0.3, 0.3, (3, ctx.V)), dtype=torch.float32, device=DEV)
    fields = H.fields_for(wl, DEV)
    p, p64, a, a_b = pressure_inputs(wl, ctx, 12)
    n = wl.grid.n
    f = tuple(torch.zeros((n[2], n[1], n[0]), dtype=torch.float32, device=DEV) for _ in range(3))
    x1, v1 = torch.empty_like(x), torch.empty_like(v)
    ctx.step(x, v, fields, x1, v1, f, p=p, accel=a)
    ctx.check_device_error()
    xs = H.to_abs(wl, H.split_state(ctx, wl, x))
    vs = [torch.tensor(t) for t in H.split_state(ctx, wl, v)]
    out = O.step(ob, xs, vs, tuple(t.double().cpu() for t in fields), H.oracle_params(wl),
                 with_spread=False, pressure=p64, accels=a_b)
    vg = H.split_state(ctx, wl, v1)
    for i in range(len(ob)):
        vo = out["v_next"][i].numpy()
        dv_o = vo - vs[i].numpy()
        store = np.linalg.norm(0.5 * np.spacing(np.abs(vo).astype(np.float32)).astype(np.float64))
        excess = max(0.0, np.linalg.norm((vg[i] - vs[i].numpy()) - dv_o) - store) / np.linalg.norm(dv_o)
        record_error(f"dv[{i}]", excess)
        assert excess <= 1e-5, (i, excess)


def soft_mixed_workload(scale=1e-5):
    """The mixed workload with its elastic constants scaled down, so that in
    a flow at rest the pressure load dominates the step's dependence on x."""
    wl = mixed_workload()
    bodies = [dataclasses.replace(b, ks=b.ks * scale, kb=b.kb * scale, ka=b.ka * scale,
                                  kA=b.kA * scale, kv=b.kv * scale) for b in wl.bodies]
    return dataclasses.replace(wl, bodies=bodies)


def oracle_vjp(wl, ob, xs, fields64, gxn_b, gvn_b, p64, a_b):
    xr = [t.clone().requires_grad_(True) for t in xs]
    vr = [torch.zeros_like(t).requires_grad_(True) for t in xs]
    for b in ob:
        for k in PARAMS:
            setattr(b, k, getattr(b, k).detach().clone().requires_grad_(True))
    out = O.step(ob, xr, vr, fields64, H.oracle_params(wl), create_graph=True, with_spread=False,
                 pressure=p64, accels=a_b)
    J = sum((out["x_next"][i] * gxn_b[i]).sum() + (out["v_next"][i] * gvn_b[i]).sum()
            for i in range(len(ob)))
    grads = torch.autograd.grad(J, xr + [getattr(b, k) for b in ob for k in PARAMS],
                                allow_unused=True)
    return [g.numpy() for g in grads[:len(ob)]], grads[len(ob):]


def test_pressure_backward_matches_oracle(record_error):
    wl = soft_mixed_workload()
    ob = H.oracle_bodies(wl)
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    rel = tie_free_state(wl, 20, scale=0.05, stretch=0.05)
    x = H.state_tensor(wl, rel)
    xs = H.to_abs(wl, H.split_state(ctx, wl, x))
    rng = np.random.default_rng(9)
    # no incoming position cotangent: gx is then the non-trivial part alone
    # (added to a unit gx', a 1e-4 part would sit at float32 resolution)
    gxn = torch.zeros((3, ctx.V), dtype=torch.float32, device=DEV)
    gvn = torch.tensor(rng.standard_normal((3, ctx.V)), dtype=torch.float32, device=DEV)
    n = wl.grid.n
    rest = tuple(torch.zeros((n[2], n[1], n[0]), dtype=torch.float32, device=DEV) for _ in range(3))
    p, p64, a, a_b = pressure_inputs(wl, ctx, 13)
    gx, gv, gp = ctx.backward(x, rest, gxn, gvn, p=p, accel=a)
    ctx.check_device_error()
    gxn_b = [torch.tensor(t) for t in H.split_state(ctx, wl, gxn)]
    gvn_b = [torch.tensor(t) for t in H.split_state(ctx, wl, gvn)]
    rest64 = tuple(t.double().cpu() for t in rest)
    ogx, ogp = oracle_vjp(wl, ob, xs, rest64, gxn_b, gvn_b, p64, a_b)
    ogx0, _ = oracle_vjp(wl, H.oracle_bodies(wl), xs, rest64, gxn_b, gvn_b, None, None)
    ggx = H.split_state(ctx, wl, gx)
    gp = gp.cpu().numpy()
    for i, b in enumerate(wl.bodies):
        d_g = ggx[i] - gxn_b[i].numpy()
        d_o = ogx[i] - gxn_b[i].numpy()
        # the pressure load carries most of the non-trivial cotangent
        share = np.linalg.norm(ogx[i] - ogx0[i]) / np.linalg.norm(d_o)
        record_error(f"pressure_share[{i}]", share)
        assert share > 0.5, (i, share)
        record_error(f"gx[{i}]", H.rel_l2(d_g, d_o))
        assert H.rel_l2(d_g, d_o) <= 1e-4, (i, H.rel_l2(d_g, d_o))
        for k, name in enumerate(PARAMS):
            g = ogp[5 * i + k]
            if g is None:
                continue
            err = abs(gp[i, k] - float(g)) / max(abs(float(g)), 1e-30)
            record_error(f"g{name}[{i}]", err)
            assert err <= 1e-4, (i, name)


def test_buoyancy_closed_form_on_gpu(record_error):
    """A closed body accelerating with a = -G in p = p0 + G.x feels exactly
    -G V in total (no flow, so no viscous load)."""
    grid = W.Grid((40, 40, 40))
    body = W._sphere_body(3, 0.18, np.array([0.47, 0.51, 0.53]), rng=np.random.default_rng(2),
                          stretch=(1.2, 1.0, 0.85))
    wl = W.Workload(name="buoy", bodies=[body], grid=grid, field={"kind": "uniform", "U": (0, 0, 0)})
    ctx = _lib.Context(wl.bodies, grid, dt=wl.dt)
    x, v = ctx.init_state()
    G = np.array([0.7, -1.3, 0.4])
    p = W.sample_pressure({"kind": "linear", "p": 0.3, "G": G}, grid, device=DEV)
    a = torch.tensor(np.repeat(-G[:, None], ctx.V, 1), dtype=torch.float32, device=DEV)
    fields = W.sample_field(wl.field, grid, device=DEV)
    _, _, Fe = ctx.interpolate(x, v, fields, U=False, F_marker=False, F_ext=True, p=p,
                               accel=a.contiguous())
    total = Fe.double().sum(1).cpu().numpy()
    rest = body.rest
    vol = float(np.einsum("ij,ij->i", rest[body.tri[:, 0]],
                          np.cross(rest[body.tri[:, 1]], rest[body.tri[:, 2]])).sum() / 6.0)
    e = np.linalg.norm(total + G * vol) / np.linalg.norm(G * vol)
    record_error("buoyancy", e)
    assert e <= 1e-5
