"""The marker kernel's direct global path against the FP64 oracle: a patch
whose stencil footprint does not fit shared memory (a coarse sphere much
larger than the grid cells: ~160 faces spanning ~10^4 grid rows) reads the
velocity from global memory, spreads with float atomics and records its
bounding box, which the next step's clear zeroes.  Two steps through the C
ABI; the second is compared (velocity increment beyond float32 storage,
spread field), so the bounding-box clear is exercised too."""
import numpy as np
import pytest
import torch

from oracle import ibm_oracle as O
from paper_1612_03399_gb300 import _lib
from paper_1612_03399_gb300 import workloads as W

import helpers as H

pytestmark = pytest.mark.gpu
DEV = "cuda"


def coarse_sphere_workload(shift=0.0):
    v, t = W.icosphere(2)                     # 320 faces: two patches of 160
    c = np.array([0.5, 0.47, 0.52]) + shift
    body = W.Body(rest=c + 0.38 * v, tri=t, origin=c, ks=1.0, kb=0.02, ka=1.0, kA=1.0, kv=1.0,
                  mass=1.0, radius=0.38)
    rng = np.random.default_rng(3)
    return W.Workload(name="coarse", bodies=[body], grid=W.Grid((72, 80, 64)),
                      field=W.fourier_modes(6, 3, 1.0, rng))


def initial_velocity(wl):
    rng = np.random.default_rng(4)
    return rng.uniform(-0.2, 0.2, (3, len(wl.bodies[0].rest))).astype(np.float32)


def tie_free_case():
    """The first of a fixed list of centre shifts for which the positions of
    the second step (x0 + dt v0 up to dt^2 a, which moves them by ~1e-6
    cells) keep 1e-4 cells from every nearest-node switch."""
    for k in range(40):
        wl = coarse_sphere_workload(shift=1e-3 * k)
        b = wl.bodies[0]
        x1 = (b.rest - b.origin).astype(np.float32) + wl.dt * initial_velocity(wl).T
        if H.tie_free(wl, [torch.tensor(x1.astype(np.float64) + b.origin)], margin=1e-4):
            return wl
    raise RuntimeError("no tie-free shift")


def test_global_path_matches_oracle(record_error):
    wl = tie_free_case()
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    fields = H.fields_for(wl, DEV)
    x, _ = ctx.init_state()
    v = torch.tensor(initial_velocity(wl), device=DEV)
    n = wl.grid.n
    f = tuple(torch.zeros((n[2], n[1], n[0]), dtype=torch.float32, device=DEV) for _ in range(3))
    x1, v1 = torch.empty_like(x), torch.empty_like(v)
    ctx.step(x, v, fields, x1, v1, f)
    assert ctx.counters()["marker_box_fallbacks"] > 0
    # the second step from the GPU's state, checked against the oracle
    xs = H.to_abs(wl, H.split_state(ctx, wl, x1))
    assert H.tie_free(wl, xs)
    x2, v2 = torch.empty_like(x), torch.empty_like(v)
    ctx.step(x1, v1, fields, x2, v2, f)
    ctx.check_device_error()
    ob = H.oracle_bodies(wl)
    vs = [torch.tensor(a) for a in H.split_state(ctx, wl, v1)]
    out = O.step(ob, xs, vs, tuple(t.double().cpu() for t in fields), H.oracle_params(wl))
    vg = H.split_state(ctx, wl, v2)[0]
    vo = out["v_next"][0].numpy()
    v0 = vs[0].numpy()
    store = np.linalg.norm(0.5 * np.spacing(np.abs(vo).astype(np.float32)).astype(np.float64))
    ev = max(0.0, np.linalg.norm((vg - v0) - (vo - v0)) - store) / np.linalg.norm(vo - v0)
    ef = H.rel_l2(torch.stack(f).cpu().numpy(), out["f"].numpy())
    record_error("dv", ev)
    record_error("f", ef)
    assert ev <= 1e-5 and ef <= 1e-5


def sheet_body(shift):
    """A coarse open sheet (~4 cells per face, clamped rim) inside the sphere,
    whose one patch spans more than 1024 grid rows."""
    rng = np.random.default_rng(7)
    sv, st, bnd = W.elliptic_sheet(0.3, 0.28, 200, rng, jitter=0.15)
    rot = W.random_rotation(rng)
    c = np.array([0.5, 0.47, 0.52]) + shift
    return W.Body(rest=c + sv @ rot.T, tri=st, origin=c, closed=False, clamped=bnd, ks=5.0,
                  kb=0.3, ka=1.0, kA=0.0, kv=0.0, mass=1.5, radius=0.3)


def test_global_path_open_sheet_and_pressure(record_error):
    """The global path with two-sided probes (open sheet), the cell-centred
    pressure and the marker-acceleration correction: traction and one step
    against the oracle."""
    for k in range(40):
        wl = coarse_sphere_workload(shift=1e-3 * k)
        wl.bodies.append(sheet_body(1e-3 * k))
        if H.tie_free(wl, [torch.tensor(b.rest) for b in wl.bodies]):
            break
    else:
        raise RuntimeError("no tie-free shift")
    sheet = wl.bodies[1]
    ext = (sheet.rest.max(0) - sheet.rest.min(0)) / np.array(wl.grid.h)
    assert (ext[1] + 4) * (ext[2] + 4) > 1024      # more (y, z) rows than shared memory holds
    ob = H.oracle_bodies(wl)
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    fields = H.fields_for(wl, DEV)
    x, _ = ctx.init_state()
    rng = np.random.default_rng(8)
    vb = []
    for b in wl.bodies:
        vv = rng.uniform(-0.2, 0.2, (len(b.rest), 3))
        if b.clamped is not None:
            vv[b.clamped] = 0.0
        vb.append(vv)
    v = H.state_tensor(wl, vb)
    spec = W.pressure_modes(12, 3, 20.0, rng)
    p = W.sample_pressure(spec, wl.grid, device=DEV, dtype=torch.float32)
    p64 = W.sample_pressure(spec, wl.grid, dtype=torch.float64)
    a = torch.tensor(rng.uniform(-20.0, 20.0, (3, ctx.V)), dtype=torch.float32, device=DEV)
    a_b = [torch.tensor(t) for t in H.split_state(ctx, wl, a)]
    _, _, Fe = ctx.interpolate(x, v, fields, U=False, F_marker=False, F_ext=True, p=p, accel=a)
    n = wl.grid.n
    f = tuple(torch.zeros((n[2], n[1], n[0]), dtype=torch.float32, device=DEV) for _ in range(3))
    x1, v1 = torch.empty_like(x), torch.empty_like(v)
    ctx.step(x, v, fields, x1, v1, f, p=p, accel=a)
    ctx.check_device_error()
    assert ctx.counters()["marker_box_fallbacks"] > 0
    xs = H.to_abs(wl, H.split_state(ctx, wl, x))
    vs = [torch.tensor(t) for t in H.split_state(ctx, wl, v)]
    out = O.step(ob, xs, vs, tuple(t.double().cpu() for t in fields), H.oracle_params(wl),
                 pressure=p64, accels=a_b)
    e = H.rel_l2(Fe.double().cpu().numpy().T, out["F_ext_face"].numpy())
    record_error("F_ext_face", e)
    assert e <= 1e-5
    vg = H.split_state(ctx, wl, v1)
    for i in range(len(wl.bodies)):
        vo = out["v_next"][i].numpy()
        v0 = vs[i].numpy()
        store = np.linalg.norm(0.5 * np.spacing(np.abs(vo).astype(np.float32)).astype(np.float64))
        ev = max(0.0, np.linalg.norm((vg[i] - v0) - (vo - v0)) - store) / np.linalg.norm(vo - v0)
        record_error(f"dv[{i}]", ev)
        assert ev <= 1e-5
    ef = H.rel_l2(torch.stack(f).cpu().numpy(), out["f"].numpy())
    record_error("f", ef)
    assert ef <= 1e-5
