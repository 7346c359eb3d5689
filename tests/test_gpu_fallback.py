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
