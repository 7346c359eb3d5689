"""The fluid phase and the coupled step on the GPU (ibm_flow_*) against the
FP64 flow oracle, through the C ABI.

Bar: relative L2 <= 1e-5 for velocities and spread forces (the float32
stencils and FFTs round at ~1e-7 relative); bodies as in the step parity
tests (positions relative to the body size, velocity changes beyond half an
ulp of float32 storage).  The pressure correction phi solves
lap(phi) = div(u*)/(alpha_l dt): the float32 divergence of a field carries
rounding ~3 eps |u|/h (three differences of size |u|/h), which the Poisson
solve (grid-scale modes scaled by ~h^2/8) and the 1/(alpha_l dt) turn into
an absolute pressure error ~3 eps |u| h/(8 alpha_l dt) per substep; the
pressure bar is relative L2 <= 1e-5 plus that floor summed over the
substeps taken.  Grids are anisotropic and not multiples of the 32 x 8
thread blocks."""
import numpy as np
import pytest
import torch

from oracle import ibm_oracle as O
from oracle import ns_oracle as N
from paper_1612_03399_gb300 import _lib
from paper_1612_03399_gb300 import workloads as W

import helpers as H
from test_gpu_parity import mixed_workload, tie_free_state

pytestmark = pytest.mark.gpu
DEV = "cuda"
DT = torch.float64


def curl_field(n, h, seed, amp=1.0):
    """Solenoidal MAC field: discrete curl of a random edge vector potential."""
    g = torch.Generator().manual_seed(seed)
    A = torch.randn((3, n[2], n[1], n[0]), generator=g, dtype=DT) * amp * min(h)
    fd = lambda f, d: (N.shift(f, d, 1) - f) / h[d]
    return torch.stack([fd(A[2], 1) - fd(A[1], 2), fd(A[0], 2) - fd(A[2], 0),
                        fd(A[1], 0) - fd(A[0], 1)])


def to_dev(t):
    return t.to(torch.float32).to(DEV).contiguous()


def fields_dev(u):
    return tuple(to_dev(u[c]) for c in range(3))


def stack_cpu(fields):
    return torch.stack([f.double().cpu() for f in fields])


def rel(a, b):
    return H.rel_l2(a.numpy(), b.numpy())


EPS32 = 2.0 ** -24


def pressure_ok(pg, po, u_max, h_min, dt, substeps):
    """rms(pg - po) <= 1e-5 rms(po) + sum over the substeps taken of
    3 eps |u|_max h_min / (8 alpha_l dt).  Returns (relative error, ok)."""
    a, b = pg.numpy(), po.numpy()
    n = np.sqrt(a.size)
    floor = sum(3 * EPS32 * u_max * h_min / (8 * N.ALPHA[l] * dt) for l in substeps)
    err = np.linalg.norm(a - b) / n
    return H.rel_l2(a, b), err <= 1e-5 * np.linalg.norm(b) / n + floor


def documented_widths(grid, nu, dt):
    """The viscous solve's path per substep by the rule the header states:
    the smallest W <= 8 with 2W + 1 <= n_d whose periodic inverse entries
    (a DFT of 1/(1 + 4c sin^2(pi k/n)), c = alpha_l dt nu / (2 h_d^2)) leave
    at most 2^-26 of their mass beyond |m| = W, the largest over the
    directions; -1 (Fourier) when some direction has none."""
    out = []
    for l in range(3):
        c_l = N.ALPHA[l] * dt * nu / 2
        wl = 0
        for d in range(3):
            n = grid.n[d]
            k = np.arange(n)
            eig = 1 + 4 * c_l / grid.h[d] ** 2 * np.sin(np.pi * k / n) ** 2
            g = np.real(np.fft.ifft(1 / eig))
            wd = next((w for w in range(9) if 2 * w + 1 <= n and
                       1 - g[0] - 2 * g[1:w + 1].sum() <= 2.0 ** -26), -1)
            wl = -1 if wd < 0 or wl < 0 else max(wl, wd)
        out.append(wl)
    return tuple(out)


@pytest.mark.parametrize("n, L, nu, widths", [
    ((40, 36, 20), (1.0, 0.9, 0.5), 0.02, (7, 4, 6)),       # real-space solves
    ((40, 36, 20), (1.0, 0.9, 0.5), 0.5, (-1, -1, -1)),     # Fourier solves
    ((40, 36, 12), (1.0, 0.9, 0.3), 0.02, (-1, 4, -1)),     # 2W + 1 > n_z in substeps 0, 2
    ((39, 36, 20), (0.975, 0.9, 0.5), 0.02, (7, 4, 6)),     # odd n_x: unpaired columns
])
def test_substeps_match_oracle(record_error, n, L, nu, widths):
    """Predictor and projection of each substep, from the same inputs, on
    both paths of the viscous solve (ragged against the real-space solve's
    32 x 16 x 32 tiles)."""
    grid = W.Grid(n, L)
    flow_o = N.Flow(grid.n, grid.L, nu=nu, dt=1e-2)
    u0 = curl_field(grid.n, grid.h, 1)
    g = torch.Generator().manual_seed(2)
    p0 = torch.randn((grid.n[2], grid.n[1], grid.n[0]), generator=g, dtype=DT)
    fl = _lib.Flow(grid, nu=flow_o.nu, dt=flow_o.dt)
    assert fl.solve_widths() == widths == documented_widths(grid, nu, flow_o.dt)
    u, p = fields_dev(u0), to_dev(p0)
    uo, po, Hp = u0.clone(), p0.clone(), None
    for l in range(3):
        fl.predict(l, u, p)
        us_o, Hp = N.predict(flow_o, l, uo, po, Hp)
        e = rel(stack_cpu(u), us_o)
        record_error(f"u*[{l}]", e)
        assert e <= 1e-5, (l, e)
        # continue both from the oracle's provisional field
        u = fields_dev(us_o)
        fl.project(l, u, p)
        uo, po = N.project(flow_o, l, us_o, po)
        eu = rel(stack_cpu(u), uo)
        ep, pok = pressure_ok(p.double().cpu(), po, float(us_o.abs().max()), min(grid.h),
                              flow_o.dt, [l])
        record_error(f"u[{l}]", eu)
        record_error(f"p[{l}]", ep)
        assert eu <= 1e-5 and pok, (l, eu, ep)
        div = N.divergence(stack_cpu(u), grid.h)
        assert float(div.abs().max()) * min(grid.h) <= 1e-5 * float(uo.abs().max())
        u, p = fields_dev(uo), to_dev(po)
    fl.close()


def test_flow_steps_match_oracle(record_error):
    """Five whole steps of the flow alone (ibm_flow_step without a context),
    from the Fourier field of the mixed workload (its discrete divergence is
    removed by the first projection)."""
    wl = mixed_workload()
    flow_o = N.Flow(wl.grid.n, wl.grid.L, nu=0.05, dt=5e-3)
    fl = _lib.Flow(wl.grid, nu=flow_o.nu, dt=flow_o.dt)
    assert fl.solve_widths() == documented_widths(wl.grid, flow_o.nu, flow_o.dt) == (7, 4, 6)
    u = tuple(f.clone() for f in H.fields_for(wl, DEV))
    p = torch.zeros_like(u[0])
    uo, po = stack_cpu(u), torch.zeros(u[0].shape, dtype=DT)
    for s in range(5):
        fl.step(u, p)
        uo, po = N.ns_step(flow_o, uo, po)
        eu = rel(stack_cpu(u), uo)
        ep, pok = pressure_ok(p.double().cpu(), po, float(uo.abs().max()), min(wl.grid.h),
                              flow_o.dt, [0, 1, 2] * (s + 1))
        record_error(f"u[{s}]", eu)
        record_error(f"p[{s}]", ep)
        assert eu <= 1e-5 and pok, (s, eu, ep)
    fl.close()


def coupled_case(seed):
    wl = mixed_workload()
    rel_x = tie_free_state(wl, seed, scale=0.03, stretch=0.03)
    rng = np.random.default_rng(seed)
    vs = []
    for b in wl.bodies:
        v = rng.uniform(-0.2, 0.2, (len(b.rest), 3))
        if b.clamped is not None:
            v[b.clamped] = 0.0
        vs.append(v)
    return wl, rel_x, vs


def test_coupled_step_matches_oracle(record_error):
    """One loosely coupled step: flow, pressure, the last substep's spread
    forcing, and the bodies."""
    wl, rel_x, vs = coupled_case(20)
    ob = H.oracle_bodies(wl)
    prm = H.oracle_params(wl)
    flow_o = N.Flow(wl.grid.n, wl.grid.L, nu=wl.mu, dt=wl.dt)
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    fl = _lib.Flow(wl.grid, nu=wl.mu, dt=wl.dt)
    # substeps 0 and 2 on the Fourier path, substep 1 in real space
    assert fl.solve_widths() == documented_widths(wl.grid, wl.mu, wl.dt) == (-1, 7, -1)
    x = H.state_tensor(wl, rel_x)
    v = H.state_tensor(wl, vs)
    u = tuple(f.clone() for f in H.fields_for(wl, DEV))
    p = torch.zeros_like(u[0])
    f = tuple(torch.empty_like(u[0]) for _ in range(3))
    x1, v1 = torch.empty_like(x), torch.empty_like(v)
    uo = stack_cpu(u)
    fl.step(u, p, ctx=ctx, x=x, v=v, x_out=x1, v_out=v1, f=f)
    ctx.check_device_error()
    xs = H.to_abs(wl, H.split_state(ctx, wl, x))
    vso = [torch.tensor(a) for a in H.split_state(ctx, wl, v)]
    xo, vo, uo, po, fo = N.coupled_step(ob, xs, vso, uo, torch.zeros(u[0].shape, dtype=DT),
                                        flow_o, prm)
    for name, a, b in (("u", stack_cpu(u), uo), ("f", stack_cpu(f), fo)):
        e = rel(a, b)
        record_error(name, e)
        assert e <= 1e-5, (name, e)
    ep, pok = pressure_ok(p.double().cpu(), po, float(uo.abs().max()), min(wl.grid.h), wl.dt,
                          [0, 1, 2])
    record_error("p", ep)
    assert pok, ep
    xg = H.split_state(ctx, wl, x1)
    vg = H.split_state(ctx, wl, v1)
    for i, b in enumerate(wl.bodies):
        size = float(np.linalg.norm(b.rest - b.origin, axis=1).max())
        xr = xo[i].numpy() - b.origin
        ex = np.linalg.norm(xg[i] - xr) / (size * np.sqrt(len(xr)))
        dvo = vo[i].numpy() - vs[i]
        store = np.linalg.norm(0.5 * np.spacing(np.abs(vo[i].numpy()).astype(np.float32)).astype(np.float64))
        ev = max(0.0, np.linalg.norm((vg[i] - vs[i]) - dvo) - store) / np.linalg.norm(dvo)
        record_error(f"x[{i}]", ex)
        record_error(f"dv[{i}]", ev)
        assert ex <= 1e-5 and ev <= 1e-5, (i, ex, ev)
    fl.close()


def test_coupled_steps_track_oracle(record_error):
    """Three coupled steps from a state whose markers stay clear of
    nearest-node switches along the oracle's trajectory."""
    steps = 3
    u_init = H.fields_for(mixed_workload(), DEV)
    for seed in range(30, 60):
        wl, rel_x, vs = coupled_case(seed)
        ob = H.oracle_bodies(wl)
        prm = H.oracle_params(wl)
        flow_o = N.Flow(wl.grid.n, wl.grid.L, nu=wl.mu, dt=wl.dt)
        xs = H.to_abs(wl, [r.astype(np.float32).astype(np.float64) for r in rel_x])
        vso = [torch.tensor(v.astype(np.float32).astype(np.float64)) for v in vs]
        uo = stack_cpu(u_init)
        po = torch.zeros(uo.shape[1:], dtype=DT)
        traj, ok = [], True
        for _ in range(steps):
            xs, vso, uo, po, _ = N.coupled_step(ob, xs, vso, uo, po, flow_o, prm)
            traj.append((xs, vso, uo, po))
            # GPU and oracle positions differ by ~1e-7 cells here, so a
            # 2e-6-cell margin keeps both on the same stencils
            if not H.tie_free(wl, xs, margin=2e-6):
                ok = False
                break
        if ok:
            break
    assert ok, "no tie-free trajectory found"
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    fl = _lib.Flow(wl.grid, nu=wl.mu, dt=wl.dt)
    x = H.state_tensor(wl, rel_x)
    v = H.state_tensor(wl, vs)
    u = tuple(t.clone() for t in u_init)
    p = torch.zeros_like(u[0])
    f = tuple(torch.empty_like(u[0]) for _ in range(3))
    for k in range(steps):
        x1, v1 = torch.empty_like(x), torch.empty_like(v)
        fl.step(u, p, ctx=ctx, x=x, v=v, x_out=x1, v_out=v1, f=f)
        x, v = x1, v1
        xs, _, uo, po = traj[k]
        eu = rel(stack_cpu(u), uo)
        ep, pok = pressure_ok(p.double().cpu(), po, float(uo.abs().max()), min(wl.grid.h), wl.dt,
                              [0, 1, 2] * (k + 1))
        record_error(f"u[{k}]", eu)
        record_error(f"p[{k}]", ep)
        assert eu <= 1e-5 and pok, (k, eu, ep)
        xg = H.split_state(ctx, wl, x)
        for i, b in enumerate(wl.bodies):
            size = float(np.linalg.norm(b.rest - b.origin, axis=1).max())
            xr = xs[i].numpy() - b.origin
            ex = np.linalg.norm(xg[i] - xr) / (size * np.sqrt(len(xr)))
            record_error(f"x[{k}][{i}]", ex)
            assert ex <= 1e-5, (k, i, ex)
    ctx.check_device_error()
    fl.close()


def test_flow_rejects_bad_use():
    wl = mixed_workload()
    with pytest.raises(_lib.IBMError):
        _lib.Flow(W.Grid((2, 8, 8)), nu=0.1, dt=1e-3)
    with pytest.raises(_lib.IBMError):
        _lib.Flow(wl.grid, nu=-1.0, dt=1e-3)
    fl = _lib.Flow(wl.grid, nu=0.1, dt=1e-3)
    u = tuple(torch.zeros((wl.grid.n[2], wl.grid.n[1], wl.grid.n[0]), device=DEV) for _ in range(3))
    p = torch.zeros_like(u[0])
    with pytest.raises(_lib.IBMError):
        fl.predict(1, u, p)              # substep 1 before substep 0
    ctx = _lib.Context(wl.bodies, wl.grid, dt=2e-3, mu=0.1)
    x, v = ctx.init_state()
    with pytest.raises(_lib.IBMError):   # dt differs from the flow's
        fl.step(u, p, ctx=ctx, x=x, v=v, x_out=torch.empty_like(x), v_out=torch.empty_like(v),
                f=tuple(torch.zeros_like(u[0]) for _ in range(3)))
    fl.close()


def test_flow_phase_times():
    """The phase-timing aid: refused before three substeps were timed, then
    13 non-negative phases whose sum is the step's device time."""
    wl, rel_x, vs = coupled_case(20)
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    fl = _lib.Flow(wl.grid, nu=wl.mu, dt=wl.dt)
    x = H.state_tensor(wl, rel_x)
    v = H.state_tensor(wl, vs)
    u = tuple(t.clone() for t in H.fields_for(wl, DEV))
    p = torch.zeros_like(u[0])
    f = tuple(torch.empty_like(u[0]) for _ in range(3))
    fl.set_phase_timing(True)
    with pytest.raises(_lib.IBMError):
        fl.phase_times()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fl.step(u, p, ctx=ctx, x=x, v=v, x_out=torch.empty_like(x), v_out=torch.empty_like(v), f=f)
    e1.record()
    e1.synchronize()
    ph = fl.phase_times()
    assert list(ph) == list(_lib.FLOW_PHASES)
    assert all(t >= 0.0 for t in ph.values())
    assert ph["rhs"] > 0 and ph["ibm_forcing"] > 0 and ph["body_force"] > 0
    assert sum(ph.values()) <= e0.elapsed_time(e1) * 1.05 + 0.05
    fl.close()


def test_coupled_step_full_size_properties(record_error):
    """The coupled benchmark's configuration (the 1000 drops on 256^3, dt at
    CFL 0.5, nu = mu = 0.01), where the oracle cannot follow (every body
    couples through the flow): after two coupled steps through the C ABI the
    velocity is discretely solenoidal to float32 rounding, every node obeys
    the symplectic update x' = x + dt v', nothing is non-finite and no marker
    patch left shared memory."""
    import bench
    wl = W.batched_drops(1000, 3, 256, seed=1)
    fields = H.fields_for(wl, DEV)
    dt = bench.cfl_dt(fields, wl.grid.h, bench.COUPLED_CFL)
    ctx = _lib.Context(wl.bodies, wl.grid, dt=dt, mu=bench.COUPLED_NU, alpha=wl.alpha,
                       patch_size=256)
    fl = _lib.Flow(wl.grid, nu=bench.COUPLED_NU, dt=dt)
    assert fl.solve_widths() == documented_widths(wl.grid, bench.COUPLED_NU, dt) == (4, 3, 3)
    u = tuple(t.clone() for t in fields)
    p = torch.zeros_like(u[0])
    f = tuple(torch.zeros_like(u[0]) for _ in range(3))
    x, v = ctx.init_state()
    for _ in range(2):
        x1, v1 = torch.empty_like(x), torch.empty_like(v)
        fl.step(u, p, ctx=ctx, x=x, v=v, x_out=x1, v_out=v1, f=f)
        x_prev, x, v = x, x1, v1
    ctx.check_device_error()
    assert ctx.counters()["marker_box_fallbacks"] == 0
    for t in (*u, p, *f, x, v):
        assert bool(torch.isfinite(t).all())
    h = wl.grid.h
    ud = [t.double() for t in u]
    div = ((torch.roll(ud[0], -1, 2) - ud[0]) / h[0] + (torch.roll(ud[1], -1, 1) - ud[1]) / h[1]
           + (torch.roll(ud[2], -1, 0) - ud[2]) / h[2])
    umax = max(float(t.abs().max()) for t in ud)
    rel_div = float(div.abs().max()) * min(h) / umax
    record_error("max|div u| h / max|u|", rel_div)
    assert rel_div <= 1e-5
    # x' = x + dt v' per node (float32 arithmetic on body-frame coordinates)
    upd = (x.double() - x_prev.double() - dt * v.double()).abs().max()
    scale = float(x_prev.abs().max())
    record_error("update residual / |x|", float(upd) / scale)
    assert float(upd) <= 4 * 2.0 ** -24 * scale
    fl.close()


def test_flow_step_full_size_matches_oracle(record_error):
    """One step of the flow alone at the coupled benchmark's configuration
    (256^3, its Fourier field, dt at CFL 0.5, nu = 0.01; real-space viscous
    solves with W = 4, 3, 3 in the benchmark's launch configuration)
    against the oracle over the whole field."""
    import bench
    wl = W.batched_drops(1000, 3, 256, seed=1)
    fields = H.fields_for(wl, DEV)
    dt = bench.cfl_dt(fields, wl.grid.h, bench.COUPLED_CFL)
    fl = _lib.Flow(wl.grid, nu=bench.COUPLED_NU, dt=dt)
    assert fl.solve_widths() == (4, 3, 3)
    flow_o = N.Flow(wl.grid.n, wl.grid.L, nu=bench.COUPLED_NU, dt=dt)
    u = tuple(t.clone() for t in fields)
    p = torch.zeros_like(u[0])
    uo = stack_cpu(u)
    fl.step(u, p)
    uo, po = N.ns_step(flow_o, uo, torch.zeros(uo.shape[1:], dtype=DT))
    eu = rel(stack_cpu(u), uo)
    ep, pok = pressure_ok(p.double().cpu(), po, float(uo.abs().max()), min(wl.grid.h), dt,
                          [0, 1, 2])
    record_error("u", eu)
    record_error("p", ep)
    assert eu <= 1e-5 and pok, (eu, ep)
    fl.close()


def test_step_and_coupled_step_keep_separate_footprints():
    """ibm_step clears the footprint of its own previous spread, the coupled
    forcing its own (it keeps a record of its own): interleaving the two on
    one context leaves each call's fields as a fresh context making only that
    call would (up to the float order of the atomic merge), with nothing
    left outside the footprint."""
    wl, rel_x, vs = coupled_case(20)

    def state():
        return H.state_tensor(wl, rel_x), H.state_tensor(wl, vs)

    def zeros3(like):
        return tuple(torch.zeros_like(like) for _ in range(3))

    fields = H.fields_for(wl, DEV)
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    fl = _lib.Flow(wl.grid, nu=wl.mu, dt=wl.dt)
    x, v = state()
    x1, v1 = torch.empty_like(x), torch.empty_like(v)
    f1 = zeros3(fields[0])
    ctx.step(x, v, fields, x1, v1, f1)
    # a coupled step from x1 into fields of its own
    u = tuple(t.clone() for t in fields)
    p = torch.zeros_like(u[0])
    f2 = zeros3(fields[0])
    x2, v2 = torch.empty_like(x), torch.empty_like(v)
    fl.step(u, p, ctx=ctx, x=x1, v=v1, x_out=x2, v_out=v2, f=f2)
    # the step again, from x1, into f1 (its previous footprint is cleared)
    x3, v3 = torch.empty_like(x), torch.empty_like(v)
    ctx.step(x1, v1, fields, x3, v3, f1)
    ctx.check_device_error()
    # references: fresh contexts, each making one of the calls
    ref = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    g1 = zeros3(fields[0])
    ref.step(x1, v1, fields, torch.empty_like(x), torch.empty_like(v), g1)
    ref2 = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    fl2 = _lib.Flow(wl.grid, nu=wl.mu, dt=wl.dt)
    u2 = tuple(t.clone() for t in fields)
    g2 = zeros3(fields[0])
    fl2.step(u2, torch.zeros_like(u2[0]), ctx=ref2, x=x1, v=v1, x_out=torch.empty_like(x),
             v_out=torch.empty_like(v), f=g2)
    ref2.check_device_error()
    for got, want in ((f1, g1), (f2, g2)):
        a, b = stack_cpu(got), stack_cpu(want)
        assert rel(a, b) <= 1e-6
        assert torch.count_nonzero(a[b == 0]) == 0
    assert rel(stack_cpu(u), stack_cpu(u2)) <= 1e-6
    for c in (ctx, ref, ref2):
        c.close()
    fl.close()
    fl2.close()
