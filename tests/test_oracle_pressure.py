"""Pins of the oracle's probe pressure with the marker-acceleration
correction, p_l = p* + h (Du/Dt).n (Sec. 2.2), against closed forms; no GPU.

In a linear pressure field p = p0 + G.x a body accelerating with a = -G (the
fluid's own acceleration for unit density) feels exactly the pressure at its
marker, because MLS reproduces linear fields and the correction h a.n cancels
the change h G.n along the probe: each face gets -p(c) n A and a closed body
the buoyancy -G V (divergence theorem, exact for flat faces and linear p).
"""
import numpy as np
import pytest
import torch

from oracle import ibm_oracle as O
from paper_1612_03399_gb300 import workloads as W

DT = torch.float64
N = 32
GRID = W.Grid((N, N, N))
G = np.array([0.7, -1.3, 0.4])
P0 = 2.5


def pressure(spec):
    return W.sample_pressure(spec, GRID, dtype=torch.float64)


def zero_velocity():
    return tuple(torch.zeros((N, N, N), dtype=DT) for _ in range(3))


def ellipsoid():
    v, t = W.icosphere(2)
    c = np.array([0.47, 0.52, 0.55])
    x = c + v * np.array([0.21, 0.17, 0.13]) @ W.random_rotation(np.random.default_rng(3))
    return O.Body(x, t, c, closed=True), torch.tensor(x, dtype=DT)


def sheet():
    rng = np.random.default_rng(5)
    sv, st, bnd = W.elliptic_sheet(0.2, 0.14, 600, rng, jitter=0.1)
    R = W.random_rotation(np.random.default_rng(7))
    c = np.array([0.5, 0.48, 0.51])
    x = c + sv @ R.T
    return O.Body(x, st, c, closed=False, clamped=bnd), torch.tensor(x, dtype=DT)


def traction(body, x, p, accel_vertex):
    C, nrm, A = O.face_geometry(x, body.tri)
    acc = None
    if accel_vertex is not None:
        a = accel_vertex
        acc = (a[body.tri[:, 0]] + a[body.tri[:, 1]] + a[body.tri[:, 2]]) / 3.0
    prm = O.Params((N, N, N))
    F = O.probe_traction(zero_velocity(), C, nrm, A, prm.n, prm.h, prm.alpha, prm.mu,
                         prm.probe_h, two_sided=not body.closed, pressure=p, accel=acc)
    return F, C, nrm, A, prm


def polyhedron_volume(x, tri):
    a, b, c = x[tri[:, 0]], x[tri[:, 1]], x[tri[:, 2]]
    return float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)


def test_accelerating_closed_body_feels_buoyancy():
    body, x = ellipsoid()
    p = pressure({"kind": "linear", "p": P0, "G": G})
    a = torch.tensor(-G, dtype=DT).expand_as(x).clone()
    F, C, nrm, A, _ = traction(body, x, p, a)
    pc = P0 + (C.numpy() @ G)
    want = -(pc * A.numpy())[:, None] * nrm.numpy()
    assert np.abs(F.numpy() - want).max() <= 1e-11 * np.abs(want).max()
    vol = polyhedron_volume(x.numpy(), body.tri.numpy())
    total = F.numpy().sum(0)
    assert np.allclose(total, -G * vol, rtol=1e-10, atol=1e-13)


def test_accelerating_open_sheet_feels_no_jump():
    body, x = sheet()
    p = pressure({"kind": "linear", "p": P0, "G": G})
    a = torch.tensor(-G, dtype=DT).expand_as(x).clone()
    F, *_ = traction(body, x, p, a)
    assert float(F.abs().max()) <= 1e-11


def test_static_open_sheet_jump_is_twice_the_probe_difference():
    """At rest (no correction) the two probe ends see p(c + h n) and
    p(c - h n): the jump is 2 h G.n and the load -2 h (G.n) n A."""
    body, x = sheet()
    p = pressure({"kind": "linear", "p": P0, "G": G})
    F, C, nrm, A, prm = traction(body, x, p, None)
    gn = nrm.numpy() @ G
    want = -(2.0 * prm.probe_h * gn * A.numpy())[:, None] * nrm.numpy()
    assert np.abs(F.numpy() - want).max() <= 1e-10 * np.abs(want).max()


def test_uniform_pressure_on_a_static_closed_body():
    body, x = ellipsoid()
    p = pressure({"kind": "uniform", "p": P0})
    F, C, nrm, A, _ = traction(body, x, p, torch.zeros_like(x))
    want = -P0 * A.numpy()[:, None] * nrm.numpy()
    assert np.abs(F.numpy() - want).max() <= 1e-12 * P0
    assert np.abs(F.numpy().sum(0)).max() <= 1e-12


def test_pressure_enters_the_node_update():
    """One step with a uniform pressure and no flow: the vertices move by the
    face loads -p0 n A / 3 over the unit mass (forces at rest are zero)."""
    body, x = ellipsoid()
    prm = O.Params((N, N, N))
    p = pressure({"kind": "uniform", "p": P0})
    out = O.step([body], [x], [torch.zeros_like(x)], zero_velocity(), prm, with_spread=False,
                 pressure=p, accels=[torch.zeros_like(x)])
    C, nrm, A = O.face_geometry(x, body.tri)
    Fv = torch.zeros_like(x)
    for k in range(3):
        Fv.index_add_(0, body.tri[:, k], -P0 * A[:, None] * nrm / 3.0)
    dv = out["v_next"][0]
    assert torch.allclose(dv, prm.dt * (Fv + out["F_int"][0]), atol=1e-14, rtol=1e-12)
