"""CUDA path vs FP64 oracle, element by element, through the C ABI.

Tolerances (float32 arithmetic against the float64 oracle on identical
inputs):
  forces, marker velocities/forces, tractions, spread fields: relative L2
  <= 1e-5; at the rest state, where forces are pure rounding, every
  component <= 10 eps32 k l0 (eps32 = 2^-23);
  positions after 100 steps: relative L2 of the body-frame positions
  <= 1e-5.
Inputs are chosen (or masked) so that no marker or probe sits within 2e-5
cells of a nearest-node switch, where float32 and float64 may pick different,
equally valid, stencils.
"""
import math

import numpy as np
import pytest
import torch

from oracle import ibm_oracle as O
from paper_1612_03399_gb300 import _lib
from paper_1612_03399_gb300 import workloads as W

import helpers as H

pytestmark = pytest.mark.gpu
DEV = "cuda"


def mixed_workload(seed=0, n=(36, 40, 32), L=(1.0, 1.1, 0.9)):
    """A closed icosphere (ragged last chunk: 320 faces), a stretched
    ellipsoid and a clamped open leaflet sheet on an anisotropic grid whose
    size is not a multiple of 8 (partial bricks)."""
    rng = np.random.default_rng(seed)
    b0 = W._sphere_body(2, 0.15, np.array([0.3, 0.42, 0.45]), ks=1.3, kb=0.05, ka=0.7, kA=1.1,
                        kv=1.9, mass=1.0)
    b1 = W._sphere_body(3, 0.12, np.array([0.68, 0.6, 0.42]), rng=rng, stretch=(1.3, 1.0, 0.8),
                        ks=0.8, kb=0.02, ka=1.0, kA=0.5, kv=1.2, mass=2.0)
    sv, st, bnd = W.elliptic_sheet(0.1, 0.07, 300, rng, jitter=0.15)
    rot = W.random_rotation(rng)
    c = np.array([0.5, 0.8, 0.6])
    b2 = W.Body(rest=c + sv @ rot.T, tri=st, origin=c, closed=False, clamped=bnd, ks=5.0, kb=0.3,
                ka=1.0, kA=0.0, kv=0.0, mass=1.5, radius=0.1)
    fld = W.fourier_modes(8, 3, 1.0, rng)
    return W.Workload(name="mixed", bodies=[b0, b1, b2], grid=W.Grid(n, L), field=fld, seed=seed)


def deformed_state(wl, seed, scale=0.05, stretch=0.05):
    xs = W.perturb_positions(wl, scale, seed, stretch=stretch)
    return H.rel_positions(wl, xs)


@pytest.fixture(scope="module")
def mixed():
    wl = mixed_workload()
    return wl, H.oracle_bodies(wl)


@pytest.mark.parametrize("patch", [0, 32, 512])
def test_internal_forces_parity(mixed, patch, record_error):
    wl, ob = mixed
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, patch_size=patch)
    rel = deformed_state(wl, 1)
    x = H.state_tensor(wl, rel)
    F, E = ctx.compute_forces(x, energy=True)
    Fg = H.split_state(ctx, wl, F)
    xs = H.to_abs(wl, H.split_state(ctx, wl, x))
    for i, b in enumerate(ob):
        Fo = b.internal_forces(xs[i]).numpy()
        record_error(f"F_int[{i}]", H.rel_l2(Fg[i], Fo))
        assert H.rel_l2(Fg[i], Fo) <= 1e-5, (i, H.rel_l2(Fg[i], Fo))
        terms = b.energy_terms(xs[i])
        for k, name in enumerate(["We", "Wb", "Wa", "WA", "Wv"]):
            ref = float(terms[name])
            got = float(E[i, k])
            assert abs(got - ref) <= 1e-5 * abs(ref) + 1e-12, (i, name, got, ref)
    ctx.check_device_error()


def test_internal_forces_at_rest_are_rounding(mixed):
    wl, ob = mixed
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt)
    x, _ = ctx.init_state()
    Fg = H.split_state(ctx, wl, ctx.compute_forces(x))
    # body-frame coordinates carry rounding ~eps32 * r, so every term's force
    # noise is ~eps32 * (stiffness) * r; allow a factor 100 over that scale
    eps = 2.0 ** -23
    for i, b in enumerate(wl.bodies):
        l0 = float(ob[i].l0.mean())
        r = float(np.linalg.norm(b.rest - b.origin, axis=1).max())
        scale = (b.ks + b.ka + b.kA + b.kv * r) * r + b.kb / l0
        assert np.abs(Fg[i]).max() <= 100 * eps * scale, (i, np.abs(Fg[i]).max(), eps * scale)


def test_body_measures_parity(mixed):
    wl, ob = mixed
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt)
    x = H.state_tensor(wl, deformed_state(wl, 2))
    m = ctx.body_measures(x).cpu().numpy()
    xs = H.to_abs(wl, H.split_state(ctx, wl, x))
    for i, b in enumerate(ob):
        _, _, Af = O.face_geometry(xs[i], b.tri)
        assert m[i, 0] == pytest.approx(float(Af.sum()), rel=1e-6)
        if b.closed:
            assert m[i, 1] == pytest.approx(float(O.enclosed_volume(xs[i], b.tri, b.origin)), rel=1e-6)
        else:
            assert m[i, 1] == 0.0


def test_interpolation_and_traction_parity(mixed, record_error):
    wl, ob = mixed
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    rng = np.random.default_rng(3)
    x = H.state_tensor(wl, deformed_state(wl, 3, scale=0.02, stretch=0.02))
    v = torch.tensor(rng.uniform(-0.5, 0.5, (3, ctx.V)), dtype=torch.float32, device=DEV)
    fields = H.fields_for(wl, DEV)
    U, Fm, Fe = ctx.interpolate(x, v, fields)
    xs = H.to_abs(wl, H.split_state(ctx, wl, x))
    vs = [torch.tensor(a) for a in H.split_state(ctx, wl, v)]
    f64 = tuple(f.double().cpu() for f in fields)
    out = O.step(ob, xs, vs, f64, H.oracle_params(wl), with_spread=False)
    keep = H.tie_mask(wl, xs)
    assert keep.mean() > 0.99
    for name, g in (("U", U), ("F_marker", Fm), ("F_ext_face", Fe)):
        gg = g.double().cpu().numpy().T[keep]
        oo = out[name].numpy()[keep]
        record_error(name, H.rel_l2(gg, oo))
        assert H.rel_l2(gg, oo) <= 1e-5, (name, H.rel_l2(gg, oo))


@pytest.mark.parametrize("variant", [1, 2])
def test_spread_parity_and_conservation(mixed, variant, record_error):
    """ibm_spread (accumulate mode) against the oracle's spread, with total
    force conserved, for both spread variants; the fields start with a
    random content that must be kept (accumulation)."""
    wl, ob = mixed
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, alpha=wl.alpha, spread_variant=variant)
    rng = np.random.default_rng(4)
    x = H.state_tensor(wl, deformed_state(wl, 4))
    xs = H.to_abs(wl, H.split_state(ctx, wl, x))
    keep = H.tie_mask(wl, xs)
    Fm = rng.standard_normal((ctx.F, 3)) * 100.0
    Fm[~keep] = 0.0
    Fm_t = torch.tensor(np.ascontiguousarray(Fm.T), dtype=torch.float32, device=DEV)
    nx, ny, nz = wl.grid.n
    g0 = torch.tensor(rng.standard_normal((3, nz, ny, nx)), dtype=torch.float32, device=DEV)
    f = tuple(g0[i].clone() for i in range(3))
    ctx.spread(x, Fm_t, f)
    ctx.check_device_error()
    f = tuple(f[i] - g0[i] for i in range(3))
    P, A = [], []
    for i, b in enumerate(ob):
        C, _, Al = O.face_geometry(xs[i], b.tri)
        P.append(C)
        A.append(Al)
    ref = O.spread(torch.tensor(Fm_t.double().cpu().numpy().T), torch.cat(P), torch.cat(A),
                   wl.grid.n, wl.grid.h, wl.alpha)
    got = torch.stack(f).double().cpu()
    # the random content (~1) is subtracted again in float32: allow its rounding
    floor = np.linalg.norm(np.spacing(np.float32(4.0))) * np.sqrt(got.numel())
    err = max(0.0, np.linalg.norm(got.numpy() - ref.numpy()) - floor) / np.linalg.norm(ref.numpy())
    record_error(f"f_v{variant}", err)
    assert err <= 1e-5
    # no net gain or loss (Eq. mls_cl), summed in float64
    dV = np.prod(wl.grid.h)
    hl = sum(wl.grid.h) / 3
    lhs = got.reshape(3, -1).sum(1).numpy() * dV
    rhs = (torch.cat(A)[:, None] * hl * torch.tensor(Fm_t.double().cpu().numpy().T)).sum(0).numpy()
    assert np.allclose(lhs, rhs, rtol=1e-5, atol=1e-6 * np.abs(rhs).max() + 1e-6 * floor * dV)


def tie_free_state(wl, seed0, **kw):
    for s in range(seed0, seed0 + 50):
        rel = deformed_state(wl, s, **kw)
        if H.tie_free(wl, H.to_abs(wl, rel)):
            return rel
    raise RuntimeError("no tie-free state found")


@pytest.mark.parametrize("forward_euler,variant,marker_patch",
                         [(False, 1, 0), (False, 2, 0), (True, 2, 0), (False, 1, 128),
                          (False, 2, 128)])
def test_step_parity(mixed, forward_euler, variant, marker_patch, record_error):
    wl, ob = mixed
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha,
                       forward_euler=forward_euler, spread_variant=variant,
                       marker_patch=marker_patch)
    assert ctx.marker_patch == (marker_patch or 256)
    rng = np.random.default_rng(5)
    rel = tie_free_state(wl, 10, scale=0.05, stretch=0.05)
    x = H.state_tensor(wl, rel)
    # float32-exact round trip: the oracle sees exactly the GPU's inputs
    xs = H.to_abs(wl, H.split_state(ctx, wl, x))
    assert H.tie_free(wl, xs)
    v = torch.tensor(rng.uniform(-0.3, 0.3, (3, ctx.V)), dtype=torch.float32, device=DEV)
    for i, b in enumerate(wl.bodies):
        if b.clamped is not None:
            o = int(ctx.v_off[i])
            v[:, o:o + len(b.rest)][:, torch.tensor(b.clamped, device=DEV)] = 0.0
    fields = H.fields_for(wl, DEV)
    nx, ny, nz = wl.grid.n
    f = tuple(torch.zeros((nz, ny, nx), dtype=torch.float32, device=DEV) for _ in range(3))
    x1, v1 = torch.empty_like(x), torch.empty_like(v)
    ctx.step(x, v, fields, x1, v1, f)
    ctx.check_device_error()
    vs = [torch.tensor(a) for a in H.split_state(ctx, wl, v)]
    f64 = tuple(ff.double().cpu() for ff in fields)
    out = O.step(ob, xs, vs, f64, H.oracle_params(wl, forward_euler=forward_euler))
    xg = H.split_state(ctx, wl, x1)
    vg = H.split_state(ctx, wl, v1)
    for i, b in enumerate(wl.bodies):
        xo = out["x_next"][i].numpy() - b.origin
        assert H.rel_l2(xg[i], xo) <= 1e-6, i
        # velocity increments carry the force error; the new velocity is stored
        # in float32, so each component also carries half an ulp of |v|
        dv_g = vg[i] - vs[i].numpy()
        vo = out["v_next"][i].numpy()
        dv_o = vo - vs[i].numpy()
        store = np.linalg.norm(0.5 * np.spacing(np.abs(vo).astype(np.float32)).astype(np.float64))
        excess = max(0.0, np.linalg.norm(dv_g - dv_o) - store) / np.linalg.norm(dv_o)
        record_error(f"dv[{i}]", excess)
        assert excess <= 1e-5, (i, excess, H.rel_l2(dv_g, dv_o))
        if b.clamped is not None:
            assert np.array_equal(xg[i][b.clamped], rel[i][b.clamped].astype(np.float32).astype(np.float64))
            assert np.all(vg[i][b.clamped] == 0)
    got = torch.stack(f).double().cpu().numpy()
    record_error("f", H.rel_l2(got, out["f"].numpy()))
    assert H.rel_l2(got, out["f"].numpy()) <= 1e-5


@pytest.mark.parametrize("variant", [1, 2])
def test_step_is_deterministic_and_clears_previous_spread(mixed, variant):
    wl, _ = mixed
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, spread_variant=variant)
    x, v = ctx.init_state()
    x = H.state_tensor(wl, deformed_state(wl, 6))
    fields = H.fields_for(wl, DEV)
    nx, ny, nz = wl.grid.n
    z = lambda: tuple(torch.zeros((nz, ny, nx), dtype=torch.float32, device=DEV) for _ in range(3))
    f = z()
    x1, v1, x2, v2 = (torch.empty_like(x) for _ in range(4))
    ctx.step(x, v, fields, x1, v1, f)
    ctx.step(x1, v1, fields, x2, v2, f)          # clears step 1's footprint first
    ctx2 = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, spread_variant=variant)
    g = z()
    y2, w2 = torch.empty_like(x), torch.empty_like(x)
    ctx2.step(x1, v1, fields, y2, w2, g)         # fresh context, zero field: step 2 only
    assert torch.equal(x2, y2) and torch.equal(v2, w2)    # bitwise: fixed summation order
    for a, b in zip(f, g):
        if variant == 2:
            assert torch.equal(a, b)                   # tile-owned: bitwise reproducible
        else:
            assert torch.allclose(a, b, rtol=1e-6, atol=1e-6 * float(b.abs().max()))


def test_single_drop_100_steps(record_error):
    """The paper's drop in frozen linear shear (Sec. 3.1 set-up): 642-node
    icosphere, 64^3 grid, 100 steps; body-frame positions within 1e-5."""
    wl = W.single_drop(level=3, n=64, steps=100)
    ob = H.oracle_bodies(wl)
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    x, v = ctx.init_state()
    fields = H.fields_for(wl, DEV)
    nx, ny, nz = wl.grid.n
    f = tuple(torch.zeros((nz, ny, nx), dtype=torch.float32, device=DEV) for _ in range(3))
    xs = H.to_abs(wl, H.split_state(ctx, wl, x))
    vs = [torch.zeros_like(xs[0])]
    xa, va = x, v
    xb, vb = torch.empty_like(x), torch.empty_like(v)
    f64 = tuple(ff.double().cpu() for ff in fields)
    prm = H.oracle_params(wl)
    for _ in range(wl.steps):
        ctx.step(xa, va, fields, xb, vb, f)
        xa, va, xb, vb = xb, vb, xa, va
        o = O.step(ob, xs, vs, f64, prm, with_spread=False)
        xs, vs = [t.detach() for t in o["x_next"]], [t.detach() for t in o["v_next"]]
    ctx.check_device_error()
    xg = H.split_state(ctx, wl, xa)[0]
    xo = xs[0].numpy() - wl.bodies[0].origin
    err = np.linalg.norm(xg - xo) / (wl.bodies[0].radius * math.sqrt(len(xo)))
    record_error("x100", err)
    assert err <= 1e-5, err
    disp = np.abs(xo - (wl.bodies[0].rest - wl.bodies[0].origin)).max()
    assert disp > 0.0


def test_rejects_bad_meshes_and_args():
    wl = mixed_workload()
    b = wl.bodies[0]
    bad = W.Body(rest=b.rest, tri=b.tri[:, [0, 2, 1]], origin=b.origin)
    with pytest.raises(_lib.IBMError) as e:
        _lib.Context([bad], wl.grid)
    assert e.value.status == 2
    flipped = b.tri.copy()
    flipped[0] = flipped[0][[0, 2, 1]]
    with pytest.raises(_lib.IBMError):
        _lib.Context([W.Body(rest=b.rest, tri=flipped, origin=b.origin)], wl.grid)
    sheet = wl.bodies[2]
    with pytest.raises(_lib.IBMError) as e:            # open sheet declared closed
        _lib.Context([W.Body(rest=sheet.rest, tri=sheet.tri, origin=sheet.origin, closed=True)],
                     wl.grid)
    assert e.value.status == 2
    with pytest.raises(_lib.IBMError):
        _lib.Context(wl.bodies, wl.grid, dt=-1.0)


def test_single_triangle_and_tiny_grid():
    """Degenerate sizes: one open triangle (3 nodes, no hinge) on the
    smallest grid; the stencil wraps in every direction."""
    rest = np.array([[0.1, 0.1, 0.1], [0.35, 0.12, 0.1], [0.2, 0.3, 0.15]])
    body = W.Body(rest=rest, tri=np.array([[0, 1, 2]], dtype=np.int32), origin=rest.mean(0),
                  closed=False, ks=2.0, kb=0.1, ka=1.0, kA=0.5, kv=0.0)
    wl = W.Workload(name="tri", bodies=[body], grid=W.Grid((4, 4, 4)),
                    field=W.fourier_modes(3, 1, 1.0, np.random.default_rng(0)))
    ob = H.oracle_bodies(wl)
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt)
    x = H.state_tensor(wl, [rest * 1.05 - body.origin * 1.05])
    xs = H.to_abs(wl, H.split_state(ctx, wl, x))
    Fg = H.split_state(ctx, wl, ctx.compute_forces(x))[0]
    assert H.rel_l2(Fg, ob[0].internal_forces(xs[0]).numpy()) <= 1e-5
    fields = H.fields_for(wl, DEV)
    v = torch.zeros_like(x)
    U, Fm, Fe = ctx.interpolate(x, v, fields)
    out = O.step(ob, xs, [torch.zeros(3, 3, dtype=torch.float64)],
                 tuple(f.double().cpu() for f in fields), H.oracle_params(wl), with_spread=False)
    if H.tie_free(wl, xs):
        assert H.rel_l2(U.double().cpu().numpy().T, out["U"].numpy()) <= 1e-5
        assert H.rel_l2(Fe.double().cpu().numpy().T, out["F_ext_face"].numpy()) <= 1e-5


def test_scalar_row_path_two_steps_with_pressure(record_error):
    """nx not a multiple of 4: rows are staged, flushed and cleared node by
    node instead of in float4 groups.  Two steps (the second clears the
    first's footprint), with a pressure field (staged like a velocity
    component), against the oracle on the second step."""
    wl = mixed_workload(n=(37, 41, 33), L=(1.0, 1.1, 0.9))
    ob = H.oracle_bodies(wl)
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    rel = tie_free_state(wl, 40, scale=0.03, stretch=0.03)
    x = H.state_tensor(wl, rel)
    v = torch.zeros_like(x)
    fields = H.fields_for(wl, DEV)
    rng = np.random.default_rng(8)
    spec = W.pressure_modes(8, 3, 5.0, rng)
    p = W.sample_pressure(spec, wl.grid, device=DEV)
    p64 = W.sample_pressure(spec, wl.grid, dtype=torch.float64)
    nx, ny, nz = wl.grid.n
    f = tuple(torch.zeros((nz, ny, nx), dtype=torch.float32, device=DEV) for _ in range(3))
    x1, v1 = torch.empty_like(x), torch.empty_like(v)
    x2, v2 = torch.empty_like(x), torch.empty_like(v)
    ctx.step(x, v, fields, x1, v1, f, p=p)
    ctx.step(x1, v1, fields, x2, v2, f, p=p)
    ctx.check_device_error()
    xs = H.to_abs(wl, H.split_state(ctx, wl, x1))
    if not H.tie_free(wl, xs):
        pytest.skip("second-step markers too close to a nearest-node switch")
    vs = [torch.tensor(a) for a in H.split_state(ctx, wl, v1)]
    out = O.step(ob, xs, vs, tuple(t.double().cpu() for t in fields), H.oracle_params(wl),
                 pressure=p64)
    vg = H.split_state(ctx, wl, v2)
    for i in range(len(ob)):
        vo = out["v_next"][i].numpy()
        dv_o = vo - vs[i].numpy()
        store = np.linalg.norm(0.5 * np.spacing(np.abs(vo).astype(np.float32)).astype(np.float64))
        excess = max(0.0, np.linalg.norm((vg[i] - vs[i].numpy()) - dv_o) - store) / np.linalg.norm(dv_o)
        record_error(f"dv[{i}]", excess)
        assert excess <= 1e-5, (i, excess)
    got = torch.stack(f).double().cpu().numpy()
    e = H.rel_l2(got, out["f"].numpy())
    record_error("f", e)
    assert e <= 1e-5


@pytest.mark.parametrize("forward_euler", [False, True])
@pytest.mark.parametrize("alias", [False, True])
def test_advance_parity(mixed, forward_euler, alias, record_error):
    """The stand-alone node update (ibm_advance; Sec. 2.3, Sec. 5 step 4):
    given F_int [3][V] and per-face F_ext [3][F], the load distribution
    F_ext^v = sum F_ext/3 and the symplectic or forward Euler update against
    the oracle's, clamped nodes fixed, outputs written in place or not."""
    wl, ob = mixed
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha,
                       forward_euler=forward_euler)
    rng = np.random.default_rng(11)
    x = H.state_tensor(wl, deformed_state(wl, 12))
    xs = H.to_abs(wl, H.split_state(ctx, wl, x))
    v = torch.tensor(rng.uniform(-0.3, 0.3, (3, ctx.V)), dtype=torch.float32, device=DEV)
    # the oracle's internal forces, and per-face loads of the same size
    Fi = H.state_tensor(wl, [b.internal_forces(xs[i]).numpy() for i, b in enumerate(ob)])
    scale = float(Fi.abs().max())
    Fe = torch.tensor(rng.uniform(-scale, scale, (3, ctx.F)), dtype=torch.float32, device=DEV)
    vs = [torch.tensor(a) for a in H.split_state(ctx, wl, v)]
    Fis = [torch.tensor(a) for a in H.split_state(ctx, wl, Fi)]
    Fes = [torch.tensor(a) for a in H.split_faces(ctx, wl, Fe)]
    if alias:
        xo, vo = x.clone(), v.clone()
        ctx.advance(xo, vo, Fi, Fe, x_out=xo, v_out=vo)
    else:
        xo, vo = ctx.advance(x, v, Fi, Fe)
    ctx.check_device_error()
    prm = H.oracle_params(wl, forward_euler=forward_euler)
    xg = H.split_state(ctx, wl, xo)
    vg = H.split_state(ctx, wl, vo)
    for i, b in enumerate(ob):
        xn, vn, _ = O.advance(b, xs[i], vs[i], Fis[i], Fes[i], prm)
        xref = xn.numpy() - wl.bodies[i].origin
        err_x = H.rel_l2(xg[i], xref)
        dv_g = vg[i] - vs[i].numpy()
        dv_o = vn.numpy() - vs[i].numpy()
        store = np.linalg.norm(0.5 * np.spacing(np.abs(vn.numpy()).astype(np.float32)).astype(np.float64))
        excess = max(0.0, np.linalg.norm(dv_g - dv_o) - store) / np.linalg.norm(dv_o)
        record_error(f"advance_x[{i}]", err_x)
        record_error(f"advance_dv[{i}]", excess)
        assert err_x <= 1e-6, (i, err_x)
        assert excess <= 1e-5, (i, excess)
        cl = wl.bodies[i].clamped
        if cl is not None and cl.any():
            x_in = H.split_state(ctx, wl, x)[i]
            assert np.array_equal(xg[i][cl], x_in[cl])
            assert np.all(vg[i][cl] == 0)


def test_tile_spread_zeroes_vacated_tiles_and_is_bitwise_reproducible(mixed):
    """Tile-owned spread (variant 2): a step at state A, then a step at state B
    (every body moved by several cells, so whole tiles empty out), leaves in
    the fields exactly what one step at B leaves in zero fields, bit for bit;
    a third context reproduces the same bits."""
    wl, _ = mixed
    rel = deformed_state(wl, 21)
    xA = H.state_tensor(wl, rel)
    shift = torch.tensor([[7.5 * wl.grid.h[0]], [-5.25 * wl.grid.h[1]], [6.0 * wl.grid.h[2]]],
                         dtype=torch.float32, device=DEV)
    xB = (xA + shift).contiguous()
    rng = np.random.default_rng(22)
    v = torch.tensor(rng.uniform(-0.3, 0.3, tuple(xA.shape)), dtype=torch.float32, device=DEV)
    fields = H.fields_for(wl, DEV)
    nx, ny, nz = wl.grid.n
    z = lambda: tuple(torch.zeros((nz, ny, nx), dtype=torch.float32, device=DEV) for _ in range(3))
    outs = []
    for k in range(3):
        ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, spread_variant=2)
        f = z()
        x1, v1 = torch.empty_like(xA), torch.empty_like(v)
        if k == 0:
            ctx.step(xA, v, fields, x1, v1, f)
            assert any(float(t.abs().sum()) > 0 for t in f)
        ctx.step(xB, v, fields, x1, v1, f)
        ctx.check_device_error()
        outs.append(f)
    for a, b, c in zip(*outs):
        assert torch.equal(a, b) and torch.equal(b, c)
    # and the fields are nonzero only near the moved bodies: the A-only
    # footprint was zeroed
    ctxA = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, spread_variant=2)
    fa = z()
    x1, v1 = torch.empty_like(xA), torch.empty_like(v)
    ctxA.step(xA, v, fields, x1, v1, fa)
    onlyA = (fa[0] != 0) & (outs[1][0] == 0)
    assert int(onlyA.sum()) > 0
    assert torch.all(outs[0][0][onlyA] == 0)
