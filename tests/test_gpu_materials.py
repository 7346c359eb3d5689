"""Van Gelder spring constants and per-face material maps (reading R18) on
the GPU, through the C ABI: forces, energies and the adjoint against the FP64
oracle; power-of-two material maps against scaled constants, bit for bit."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import ibm_oracle as O
from paper_1612_03399_gb300 import _lib

import helpers as H
from test_gpu_adjoint import oracle_vjp
from test_gpu_parity import deformed_state, mixed_workload, tie_free_state

pytestmark = pytest.mark.gpu
DEV = "cuda"
PARAMS = ["ks", "kb", "ka", "kA", "kv"]


def material_workload(seed=0):
    """The mixed workload with a two-region material on the sphere, van
    Gelder springs on the ellipsoid and both on the open sheet."""
    wl = mixed_workload()
    rng = np.random.default_rng(seed)
    b0, b1, b2 = wl.bodies
    cen0 = b0.rest[b0.tri].mean(1)
    m0 = np.where((cen0[:, 2] > b0.origin[2])[:, None], [2.5, 0.4, 3.0], [1.0, 1.0, 1.0])
    m2 = rng.uniform(0.5, 2.0, (len(b2.tri), 3))
    bodies = [dataclasses.replace(b0, face_material=m0.astype(np.float32)),
              dataclasses.replace(b1, spring_model=1, ks=0.8),
              dataclasses.replace(b2, spring_model=1, face_material=m2.astype(np.float32))]
    return dataclasses.replace(wl, bodies=bodies)


def test_forces_and_energies_with_materials(record_error):
    wl = material_workload()
    ob = H.oracle_bodies(wl)
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt)
    x = H.state_tensor(wl, deformed_state(wl, 1))
    F, E = ctx.compute_forces(x, energy=True)
    Fg = H.split_state(ctx, wl, F)
    xs = H.to_abs(wl, H.split_state(ctx, wl, x))
    for i, b in enumerate(ob):
        Fo = b.internal_forces(xs[i]).numpy()
        e = H.rel_l2(Fg[i], Fo)
        record_error(f"F_int[{i}]", e)
        assert e <= 1e-5, (i, e)
        terms = b.energy_terms(xs[i])
        for k, name in enumerate(["We", "Wb", "Wa", "WA", "Wv"]):
            ref = float(terms[name])
            assert abs(float(E[i, k]) - ref) <= 1e-5 * abs(ref) + 1e-12, (i, name)


def test_power_of_two_materials_equal_scaled_constants_bitwise():
    wl = mixed_workload()
    mat = [np.tile(np.float32([2.0, 4.0, 0.5]), (len(b.tri), 1)) for b in wl.bodies]
    wl_m = dataclasses.replace(wl, bodies=[dataclasses.replace(b, face_material=m)
                                           for b, m in zip(wl.bodies, mat)])
    wl_k = dataclasses.replace(wl, bodies=[dataclasses.replace(b, ks=2 * b.ks, kb=4 * b.kb,
                                                               ka=0.5 * b.ka)
                                           for b in wl.bodies])
    x = H.state_tensor(wl, deformed_state(wl, 2))
    Fm = _lib.Context(wl_m.bodies, wl.grid, dt=wl.dt).compute_forces(x)
    Fk = _lib.Context(wl_k.bodies, wl.grid, dt=wl.dt).compute_forces(x)
    assert torch.equal(Fm, Fk)


def test_backward_with_materials_matches_oracle(record_error):
    wl = material_workload()
    ob = H.oracle_bodies(wl)
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    rel = tie_free_state(wl, 20, scale=0.05, stretch=0.05)
    x = H.state_tensor(wl, rel)
    xs = H.to_abs(wl, H.split_state(ctx, wl, x))
    rng = np.random.default_rng(9)
    gxn = torch.tensor(rng.standard_normal((3, ctx.V)), dtype=torch.float32, device=DEV)
    gvn = torch.tensor(rng.standard_normal((3, ctx.V)), dtype=torch.float32, device=DEV)
    fields = H.fields_for(wl, DEV)
    gx, gv, gp = ctx.backward(x, fields, gxn, gvn)
    ctx.check_device_error()
    vs = [torch.zeros_like(t) for t in xs]
    gxn_b = [torch.tensor(a) for a in H.split_state(ctx, wl, gxn)]
    gvn_b = [torch.tensor(a) for a in H.split_state(ctx, wl, gvn)]
    ogx, ogv, ogp = oracle_vjp(wl, ob, xs, vs, tuple(f.double().cpu() for f in fields), gxn_b,
                               gvn_b)
    ggx = H.split_state(ctx, wl, gx)
    gp = gp.cpu().numpy()
    for i, b in enumerate(wl.bodies):
        d_g = ggx[i] - gxn_b[i].numpy()
        d_o = ogx[i] - gxn_b[i].numpy()
        record_error(f"gx[{i}]", H.rel_l2(d_g, d_o))
        assert H.rel_l2(d_g, d_o) <= 1e-4, (i, H.rel_l2(d_g, d_o))
        for k, name in enumerate(PARAMS):
            if not b.closed and name == "kv":
                continue
            err = abs(gp[i, k] - ogp[i, k]) / max(abs(ogp[i, k]), 1e-30)
            record_error(f"g{name}[{i}]", err)
            assert err <= 1e-4, (i, name, gp[i, k], ogp[i, k])
