"""Parity at the benchmarked size and launch configuration: 1000 icosphere
drops on a 512^3 grid, one ibm_step exactly as bench.py runs it.  The oracle
recomputes a sample of well-separated bodies on the same grid and field
(their supports overlap no other body's, so the spread force on their
footprint is theirs alone); the whole-field total force is checked against
the markers' forces (no net gain or loss, Eq. mls_cl)."""
import numpy as np
import pytest
import torch

from oracle import ibm_oracle as O
from paper_1612_03399_gb300 import _lib
from paper_1612_03399_gb300 import workloads as W

import helpers as H

pytestmark = pytest.mark.gpu
DEV = "cuda"


def isolated(wl, k, min_gap_cells=10):
    c = np.array([b.origin for b in wl.bodies])
    r = np.array([b.radius for b in wl.bodies])
    h = wl.grid.h[0]
    d = c[:, None, :] - c[None, :, :]
    d -= np.round(d)
    gap = np.linalg.norm(d, axis=2) - r[:, None] - r[None, :]
    np.fill_diagonal(gap, np.inf)
    ok = np.where(gap.min(1) > min_gap_cells * h)[0]
    return ok[:k]


def test_full_size_step_sampled_parity(record_error):
    wl = W.batched_drops(1000, 3, 512, seed=1)
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    fields = H.fields_for(wl, DEV)
    x, v = ctx.init_state()
    rng = np.random.default_rng(0)
    x += torch.tensor(rng.uniform(-1e-4, 1e-4, tuple(x.shape)), dtype=torch.float32, device=DEV)
    v = torch.tensor(rng.uniform(-0.2, 0.2, tuple(v.shape)), dtype=torch.float32, device=DEV)
    n = wl.grid.n
    f = tuple(torch.zeros((n[2], n[1], n[0]), dtype=torch.float32, device=DEV) for _ in range(3))
    x1, v1 = torch.empty_like(x), torch.empty_like(v)
    ctx.step(x, v, fields, x1, v1, f)
    ctx.check_device_error()
    # whole-field conservation: sum_k dV f^k = sum_l dV^l F_l
    _, Fm, _ = ctx.interpolate(x, v, fields, U=False, F_marker=True, F_ext=False)
    A = torch.zeros(ctx.F, dtype=torch.float64, device=DEV)
    xs_all = H.split_state(ctx, wl, x)
    areas = []
    for i, b in enumerate(wl.bodies):
        p = xs_all[i]
        areas.append(0.5 * np.linalg.norm(np.cross(p[b.tri[:, 1]] - p[b.tri[:, 0]],
                                                   p[b.tri[:, 2]] - p[b.tri[:, 0]]), axis=1))
    A = torch.tensor(np.concatenate(areas), device=DEV)
    hl = sum(wl.grid.h) / 3
    dV = float(np.prod(wl.grid.h))
    rhs = (A[None, :] * hl * Fm.double()).sum(1)
    lhs = torch.stack([fi.double().sum() for fi in f]) * dV
    cons = float((lhs - rhs).abs().max() / rhs.abs().max())
    record_error("conservation", cons)
    assert cons <= 1e-5
    # sampled bodies, recomputed by the oracle alone
    pick = [int(i) for i in isolated(wl, 3)]
    assert len(pick) == 3
    sub = W.Workload(name="sample", bodies=[wl.bodies[i] for i in pick], grid=wl.grid,
                     field=wl.field, dt=wl.dt)
    ob = H.oracle_bodies(sub)
    xs = [torch.tensor(xs_all[i] + wl.bodies[i].origin) for i in pick]
    vall = H.split_state(ctx, wl, v)
    vs = [torch.tensor(vall[i]) for i in pick]
    assert H.tie_free(sub, xs)
    f64 = tuple(fi.double().cpu() for fi in fields)
    out = O.step(ob, xs, vs, f64, H.oracle_params(sub))
    xg, vg = H.split_state(ctx, wl, x1), H.split_state(ctx, wl, v1)
    for j, i in enumerate(pick):
        xo = out["x_next"][j].numpy() - wl.bodies[i].origin
        assert H.rel_l2(xg[i], xo) <= 1e-6
        vo = out["v_next"][j].numpy()
        dv_o = vo - vs[j].numpy()
        store = np.linalg.norm(0.5 * np.spacing(np.abs(vo).astype(np.float32)).astype(np.float64))
        excess = max(0.0, np.linalg.norm((vg[i] - vs[j].numpy()) - dv_o) - store) / np.linalg.norm(dv_o)
        record_error(f"dv[{i}]", excess)
        assert excess <= 1e-5
    fo = out["f"].numpy()
    mask = np.abs(fo).sum(0) > 0
    got = torch.stack(f).cpu().numpy()
    e = H.rel_l2(got[:, mask], fo[:, mask])
    record_error("f_sampled", e)
    assert e <= 1e-5
