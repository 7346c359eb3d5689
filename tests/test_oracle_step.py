"""Pins of the oracle's whole step (Sec. 5 steps 1-4 with a frozen flow),
node update and Taylor deformation; no GPU."""
import math

import numpy as np
import pytest
import torch

from oracle import ibm_oracle as O
from paper_1612_03399_gb300 import workloads as W

DT = torch.float64


def small_drop(level=2, n=24, r=0.2, centre=(0.5, 0.5, 0.5), **k):
    v, t = W.icosphere(level)
    c = np.array(centre)
    return O.Body(c + r * v, t, c, **k), O.Params((n, n, n))


def fields_of(spec, n):
    nn = tuple(n) if isinstance(n, tuple) else (n, n, n)
    return tuple(f.to(DT) for f in W.sample_field(spec, W.Grid(nn), dtype=torch.float64))


def test_uniform_flow_rigid_translation():
    """Body at rest shape moving with a uniform flow U0: marker forces
    F = (V^b - U)/dt vanish (MLS reproduces constants), the traction is zero
    and every node moves by dt U0 per step."""
    b, prm = small_drop(ks=1.0, kb=0.1)
    U0 = (0.3, -0.2, 0.5)
    f = fields_of({"kind": "uniform", "U": U0}, prm.n)
    x = b.rest.clone()
    v = torch.tensor(U0, dtype=DT).expand_as(x).clone()
    out = O.step([b], [x], [v], f, prm)
    assert float(out["F_marker"].abs().max()) < 1e-9
    assert float(out["F_ext_face"].abs().max()) < 1e-12
    assert float(out["f"].abs().max()) < 1e-7
    assert torch.allclose(out["x_next"][0], x + prm.dt * torch.tensor(U0, dtype=DT), atol=1e-15)


def test_constant_force_symplectic_euler_closed_form():
    """Constant acceleration a on free nodes: symplectic Euler gives
    v_n = n dt a and x_n = x_0 + dt^2 a n(n+1)/2; forward Euler gives
    x_n = x_0 + dt^2 a n(n-1)/2.  A closed body with zero elastic constants
    in a linear flow sees a traction fixed by its normals, which barely turn
    over a few short steps, so each node's acceleration is constant."""
    b, prm = small_drop(ks=0.0, kb=0.0, ka=0.0, kA=0.0, kv=0.0, mass=2.0)
    prm = O.Params(prm.n, dt=1e-3)
    G = np.array([[0, 0.4, 0], [0.1, 0, 0], [0, 0, -0.1]])
    f = fields_of({"kind": "linear", "G": G, "c": [0, 0, 0]}, prm.n)
    x0 = b.rest.clone()
    v0 = torch.zeros_like(x0)
    a = O.step([b], [x0], [v0], f, prm)["F_ext_vertex"][0] / 2.0
    x, v = x0, v0
    nsteps = 5
    for _ in range(nsteps):
        out = O.step([b], [x], [v], f, prm, with_spread=False)
        x, v = out["x_next"][0], out["v_next"][0]
    tol = 1e-6 * float(a.abs().max())
    assert torch.allclose(v, nsteps * prm.dt * a, rtol=1e-5, atol=tol * prm.dt)
    assert torch.allclose(x - x0, prm.dt ** 2 * a * nsteps * (nsteps + 1) / 2, rtol=1e-5,
                          atol=tol * prm.dt ** 2)
    pf = O.Params(prm.n, dt=1e-3, forward_euler=True)
    x, v = x0, v0
    for _ in range(nsteps):
        out = O.step([b], [x], [v], f, pf, with_spread=False)
        x, v = out["x_next"][0], out["v_next"][0]
    assert torch.allclose(x - x0, prm.dt ** 2 * a * nsteps * (nsteps - 1) / 2, rtol=1e-5,
                          atol=tol * prm.dt ** 2)


def test_closed_body_net_traction_zero_in_linear_flow():
    """For a linear velocity field grad u is constant, so the total traction
    mu (G + G^T) sum_f n_f A_f vanishes on a closed surface
    (sum_f n_f A_f = 0)."""
    b, prm = small_drop(level=3, n=32, r=0.25)
    G = np.array([[0.2, 1.0, 0], [0, -0.3, 0.5], [0.4, 0, 0.1]])
    f = fields_of({"kind": "linear", "G": G, "c": [0.1, 0, 0]}, prm.n)
    out = O.step([b], [b.rest.clone()], [torch.zeros_like(b.rest)], f, prm, with_spread=False)
    Fe = out["F_ext_face"]
    assert float(Fe.sum(0).abs().max()) < 1e-12 * float(Fe.abs().max()) * len(Fe)
    # and the per-face traction is the closed form mu (G + G^T) n A
    C, nrm, A = O.face_geometry(b.rest, b.tri)
    ref = (nrm @ torch.tensor(G + G.T)) * A[:, None]
    assert torch.allclose(Fe, ref, atol=1e-12)


def test_clamped_nodes_stay_fixed():
    rng = np.random.default_rng(2)
    v, t, bnd = W.elliptic_sheet(0.2, 0.15, 400, rng, jitter=0.2)
    c = np.array([0.5, 0.5, 0.5])
    b = O.Body(c + v, t, c, closed=False, clamped=bnd, ks=5, kb=1, ka=1, kA=0, kv=0)
    prm = O.Params((24, 24, 24))
    f = fields_of(W.fourier_modes(8, 3, 1.0, rng), 24)
    x = b.rest + torch.tensor(rng.uniform(-1e-3, 1e-3, b.rest.shape)) * (~b.clamped)[:, None]
    vv = torch.zeros_like(x)
    for _ in range(3):
        out = O.step([b], [x], [vv], f, prm, with_spread=False)
        x, vv = out["x_next"][0], out["v_next"][0]
    assert torch.equal(x[b.clamped], b.rest[b.clamped])
    assert float(vv[b.clamped].abs().max()) == 0.0
    assert float(vv[~b.clamped].abs().max()) > 0.0


def test_periodic_shift_covariance():
    """Shifting a body and the field by whole cells shifts every output:
    positions by the same vector, force fields by the same roll."""
    rng = np.random.default_rng(3)
    n = 20
    b0, prm = small_drop(level=2, n=n, r=0.15, centre=(0.3, 0.45, 0.6), ks=1.2, kb=0.05)
    spec = W.fourier_modes(6, 3, 1.0, rng)
    f = fields_of(spec, n)
    x0 = b0.rest + torch.tensor(rng.uniform(-2e-3, 2e-3, b0.rest.shape))
    v0 = torch.tensor(rng.uniform(-0.1, 0.1, b0.rest.shape))
    out0 = O.step([b0], [x0], [v0], f, prm)
    s = np.array([3, -2, 5])
    shift = torch.tensor(s / n, dtype=DT)
    b1 = O.Body(b0.rest.numpy() + s / n, b0.tri.numpy(), b0.origin.numpy() + s / n, ks=1.2, kb=0.05)
    f1 = tuple(torch.roll(fi, shifts=(int(s[2]), int(s[1]), int(s[0])), dims=(0, 1, 2)) for fi in f)
    out1 = O.step([b1], [x0 + shift], [v0], f1, prm)
    assert torch.allclose(out1["x_next"][0] - shift, out0["x_next"][0], atol=1e-14)
    assert torch.allclose(out1["F_ext_face"], out0["F_ext_face"], rtol=1e-10, atol=1e-13)
    rolled = torch.roll(out0["f"], shifts=(int(s[2]), int(s[1]), int(s[0])), dims=(1, 2, 3))
    assert torch.allclose(out1["f"], rolled, rtol=1e-9, atol=1e-9 * float(out0["f"].abs().max()))


def test_taylor_deformation_sphere_and_ellipsoid():
    """An icosphere has icosahedral symmetry, so its second-moment tensor is
    isotropic and D = 0.  A linear map diag(a, b, c) turns that tensor into
    k diag(a^2, b^2, c^2), so an icosphere mapped onto an ellipsoid has
    D = (a - c)/(a + c) exactly at every level; its volume and moments tend
    to the solid ellipsoid's as the mesh is refined."""
    v, t = W.icosphere(3)
    tt = torch.tensor(t, dtype=torch.long)
    D0 = O.taylor_deformation(torch.tensor(0.3 * v), tt, torch.zeros(3, dtype=DT))
    assert abs(float(D0)) < 1e-12
    ax = np.array([0.33, 0.25, 0.2])
    exact = (0.33 - 0.2) / (0.33 + 0.2)
    errs = []
    for level in (2, 3, 4):
        v, t = W.icosphere(level)
        D = O.taylor_deformation(torch.tensor(v * ax + 0.1), torch.tensor(t, dtype=torch.long),
                                 torch.tensor([0.1, 0.1, 0.1], dtype=DT))
        errs.append(abs(float(D) - exact))
    assert max(errs) < 1e-13
    # volume second moment of a solid ellipsoid: a_i^2 / 5
    V, M = O.second_moment(torch.tensor(v * ax), torch.tensor(t, dtype=torch.long), torch.zeros(3, dtype=DT))
    assert float(V) == pytest.approx(4 / 3 * math.pi * ax.prod(), rel=3e-3)
    assert np.allclose(np.diag(M.numpy()), ax ** 2 / 5, rtol=1e-2)


def test_step_gradient_flows_to_constants():
    """The oracle step is differentiable end to end (the FP64 adjoint used
    to check the GPU adjoint): d x_next / d k_s is finite and matches a
    central difference."""
    b, prm = small_drop(level=1, n=16, r=0.2, ks=1.0)
    rng = np.random.default_rng(4)
    f = fields_of(W.fourier_modes(4, 2, 1.0, rng), 16)
    x0 = b.rest + torch.tensor(rng.uniform(-5e-3, 5e-3, b.rest.shape))
    v0 = torch.zeros_like(x0)
    b.ks = b.ks.clone().requires_grad_(True)
    out = O.step([b], [x0], [v0], f, prm, create_graph=True, with_spread=False)
    w = torch.tensor(rng.standard_normal(x0.shape))
    J = ((out["x_next"][0] - x0) * w).sum()
    (g,) = torch.autograd.grad(J, b.ks)
    h = 0.25          # x_next is affine in k_s, so the central difference is exact
    vals = []
    for s in (1, -1):
        bb, _ = small_drop(level=1, n=16, r=0.2, ks=1.0 + s * h)
        vals.append(float(((O.step([bb], [x0], [v0], f, prm, with_spread=False)["x_next"][0] - x0) * w).sum()))
    assert float(g) == pytest.approx((vals[0] - vals[1]) / (2 * h), rel=1e-9)


def test_rollout_loss_gradient_vs_central_differences():
    """Reverse mode of the oracle through several steps and the Taylor
    deformation equals central differences (h = 1e-4 relative) of the same
    float64 loss in k_s and k_b: the FP64 reference the GPU adjoint is held to."""
    v, t = W.icosphere(1)
    c = np.array([0.5, 0.45, 0.5])
    rest = c + 0.15 * v * np.array([1.1, 1.0, 0.95])
    f = fields_of({"kind": "shear"}, 16)
    prm = O.Params((16, 16, 16), dt=5e-3)

    def loss_of(ks, kb, grad=False):
        b = O.Body(rest, t, c, ks=1.0, kb=0.02, mass=1e-3)
        b.ks = torch.tensor(ks, dtype=DT, requires_grad=grad)
        b.kb = torch.tensor(kb, dtype=DT, requires_grad=grad)
        x, vv = [b.rest.clone()], [torch.zeros_like(b.rest)]
        for _ in range(4):
            out = O.step([b], x, vv, f, prm, create_graph=grad, with_spread=False)
            x, vv = out["x_next"], out["v_next"]
        L = (O.taylor_deformation(x[0], b.tri, b.origin) - 0.02) ** 2
        if grad:
            return torch.autograd.grad(L, [b.ks, b.kb])
        return float(L)

    g_ks, g_kb = loss_of(1.0, 0.02, grad=True)
    for val, g, which in ((1.0, g_ks, 0), (0.02, g_kb, 1)):
        h = 1e-4 * val
        args_p = [1.0, 0.02]
        args_m = [1.0, 0.02]
        args_p[which] += h
        args_m[which] -= h
        fd = (loss_of(*args_p) - loss_of(*args_m)) / (2 * h)
        assert float(g) == pytest.approx(fd, rel=1e-4)
