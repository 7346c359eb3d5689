"""Pins of the oracle's MLS transfer function, probe gradient and spreading
(Sec. 2.2, Eqs. mls..mls_cl); no GPU."""
import math

import numpy as np
import pytest
import torch

from oracle import ibm_oracle as O

DT = torch.float64
N = (16, 12, 20)
L = (1.0, 0.75, 1.25)
H = tuple(L[d] / N[d] for d in range(3))


def points(m=200, seed=0):
    rng = np.random.default_rng(seed)
    return torch.tensor(rng.uniform(-0.3, 1.4, (m, 3)) * np.array(L))


@pytest.mark.parametrize("comp", [0, 1, 2])
def test_partition_of_unity_and_linear_reproduction(comp):
    """A linear basis makes MLS reproduce constants and linear functions
    exactly (Sec. 2.2): sum phi = 1, sum phi_k x^k = x."""
    P = points()
    flat, pos, _ = O.mls_stencil(P, comp, N, H)
    _, phi = O.mls_shape(P, comp, N, H, 0.3)
    assert torch.allclose(phi.sum(1), torch.ones(len(P), dtype=DT), atol=1e-13)
    rec = (phi[..., None] * pos).sum(1)
    assert torch.allclose(rec, P, atol=1e-13)


def closed_form_phi(P, comp, alpha):
    """Independent closed form of the MLS shape functions for a weight that
    factorises over directions, W = prod_d w_d (reading R3): with per-direction
    normalised weights wh_d, mean mu_d and variance s2_d of the node offsets,
    the moment matrix is m0 [[1, mu^T], [mu, diag(s2) + mu mu^T]] and
    phi_k = prod_d wh_d(k_d) * (1 - sum_d mu_d (delta_kd - mu_d) / s2_d)."""
    off = np.array(O.MAC_OFFSET[comp])
    out = []
    for p in P.numpy():
        t = p / np.array(H) - off
        ic = np.floor(t + 0.5)
        per = []
        for d in range(3):
            delta = (ic[d] + np.array([-1.0, 0.0, 1.0]) - t[d])          # in cells
            w = np.exp(-(delta / 1.5) ** 2 / alpha ** 2)
            wh = w / w.sum()
            mu = (wh * delta).sum()
            s2 = (wh * (delta - mu) ** 2).sum()
            per.append((wh, mu * (delta - mu) / s2))
        phi = np.zeros(27)
        k = 0
        for sz in range(3):
            for sy in range(3):
                for sx in range(3):
                    s = (sx, sy, sz)
                    prod = per[0][0][sx] * per[1][0][sy] * per[2][0][sz]
                    phi[k] = prod * (1.0 - sum(per[d][1][s[d]] for d in range(3)))
                    k += 1
        out.append(phi)
    return torch.tensor(np.array(out))


@pytest.mark.parametrize("comp", [0, 1, 2])
@pytest.mark.parametrize("alpha", [0.3, 0.6])
def test_general_solve_equals_closed_form(comp, alpha):
    P = points(60, seed=comp)
    _, phi = O.mls_shape(P, comp, N, H, alpha)
    assert torch.allclose(phi, closed_form_phi(P, comp, alpha), rtol=1e-11, atol=1e-13)


def test_stencil_nearest_node_and_periodic_wrap():
    """Centre node = nearest node of the component lattice; indices wrap."""
    P = torch.tensor([[0.0, 0.0, 0.0], [L[0] - 1e-9, 0.5 * H[1], 0.49 * H[2]]], dtype=DT)
    flat, pos, centre = O.mls_stencil(P, 0, N, H)
    # u lattice: x at i h, y at (j + 1/2) h, z at (k + 1/2) h
    assert torch.allclose(centre[0], torch.tensor([0.0, 0.5 * H[1], 0.5 * H[2]], dtype=DT))
    assert torch.allclose(centre[1], torch.tensor([L[0], 0.5 * H[1], 0.5 * H[2]], dtype=DT))
    # second point: x node index n_x wraps to 0
    assert int(flat[1, 13]) == 0
    assert int(flat[0, 0]) == ((N[2] - 1) * N[1] + (N[1] - 1)) * N[0] + (N[0] - 1)


def linear_field(comp, G, c):
    off = O.MAC_OFFSET[comp]
    x = (torch.arange(N[0], dtype=DT) + off[0]) * H[0]
    y = (torch.arange(N[1], dtype=DT) + off[1]) * H[1]
    z = (torch.arange(N[2], dtype=DT) + off[2]) * H[2]
    return (c + G[0] * x.view(1, 1, -1) + G[1] * y.view(1, -1, 1) + G[2] * z.view(-1, 1, 1)).expand(
        N[2], N[1], N[0]).contiguous()


@pytest.mark.parametrize("comp", [0, 1, 2])
def test_linear_field_value_and_gradient_exact(comp):
    """Away from the periodic seam a linear field is interpolated exactly and
    its full-derivative MLS gradient is the exact gradient."""
    rng = np.random.default_rng(3)
    G, c = rng.standard_normal(3), 0.7
    f = linear_field(comp, G, c)
    P = torch.tensor(rng.uniform(0.2, 0.8, (50, 3)) * np.array(L))
    val = O.interpolate(f, P, comp, N, H, 0.3)
    assert torch.allclose(val, c + P @ torch.tensor(G), atol=1e-12)
    grad = O.interpolate_gradient(f, P, comp, N, H, 0.3)
    assert torch.allclose(grad, torch.tensor(G).expand(50, 3), atol=1e-10)


@pytest.mark.parametrize("comp", [0, 1, 2])
def test_full_derivative_vs_central_differences(comp):
    """d phi / dx equals the central difference of phi(x) with the stencil
    held fixed (points kept away from half-cell switches)."""
    rng = np.random.default_rng(7 + comp)
    off = np.array(O.MAC_OFFSET[comp])
    cells = rng.integers(2, 8, (30, 3))
    frac = rng.uniform(-0.4, 0.4, (30, 3))
    P = torch.tensor((cells + off + frac) * np.array(H))
    _, phi, dphi = O.mls_shape(P, comp, N, H, 0.3, with_grad=True)
    eps = 1e-6
    for e in range(3):
        dp = torch.zeros(3, dtype=DT)
        dp[e] = eps * H[e]
        _, pp = O.mls_shape(P + dp, comp, N, H, 0.3)
        _, pm = O.mls_shape(P - dp, comp, N, H, 0.3)
        fd = (pp - pm) / (2 * eps * H[e])
        assert torch.allclose(dphi[..., e], fd, rtol=1e-6, atol=1e-6 / H[e])


def test_spread_conserves_total_force_and_cl_closed_form():
    """Eq. mls_cl: no net gain or loss, sum_k dV f^k = sum_l dV^l F_l, and on
    a uniform grid c_l = A_l (hx + hy + hz)/3 / (hx hy hz)."""
    rng = np.random.default_rng(11)
    P = points(80, seed=4)
    F = torch.tensor(rng.standard_normal((80, 3)))
    A = torch.tensor(rng.uniform(0.1, 1.0, 80)) * H[0] * H[1]
    f = O.spread(F, P, A, N, H, 0.3)
    dV = H[0] * H[1] * H[2]
    hl = sum(H) / 3.0
    lhs = f.reshape(3, -1).sum(1) * dV
    rhs = (A[:, None] * hl * F).sum(0)
    assert torch.allclose(lhs, rhs, rtol=1e-12, atol=1e-15)
    # one marker: f = c_l phi F with the closed-form c_l
    f1 = O.spread(F[:1], P[:1], A[:1], N, H, 0.3)
    flat, phi = O.mls_shape(P[:1], 1, N, H, 0.3)
    cl = float(A[0]) * hl / dV
    got = f1[1].reshape(-1)[flat[0]]
    assert torch.allclose(got, cl * phi[0] * F[0, 1], rtol=1e-12)


def test_spread_is_weighted_transpose_of_interpolation():
    """sum_k dV f^k g^k = sum_l dV^l F_l . interp(g)_l for any grid field g."""
    rng = np.random.default_rng(12)
    P = points(40, seed=5)
    F = torch.tensor(rng.standard_normal((40, 3)))
    A = torch.tensor(rng.uniform(0.1, 1.0, 40)) * H[0] * H[1]
    f = O.spread(F, P, A, N, H, 0.3)
    g = torch.tensor(rng.standard_normal((3, N[2], N[1], N[0])))
    dV = H[0] * H[1] * H[2]
    lhs = (f * g).sum() * dV
    interp = torch.stack([O.interpolate(g[i], P, i, N, H, 0.3) for i in range(3)], 1)
    rhs = (A[:, None] * (sum(H) / 3.0) * F * interp).sum()
    assert float(lhs) == pytest.approx(float(rhs), rel=1e-12)


def test_probe_traction_closed_forms():
    """Linear shear u = (g z, 0, 0) on a flat sheet with normal +z:
    tau = mu g (e_x e_z^T + e_z e_x^T), so a one-sided probe gives
    F_ext = mu g A e_x and a two-sided one (tau+ - tau-) . n = 0."""
    g, mu = 0.8, 1.3
    G = np.zeros((3, 3))
    G[0, 2] = g
    fields = [linear_field(i, G[i], 0.0) for i in range(3)]
    C = torch.tensor([[0.5, 0.4, 0.6], [0.3, 0.35, 0.55]], dtype=DT)
    nrm = torch.tensor([[0.0, 0.0, 1.0]] * 2, dtype=DT)
    A = torch.tensor([0.01, 0.02], dtype=DT)
    F1 = O.probe_traction(fields, C, nrm, A, N, H, 0.3, mu, sum(H) / 3, two_sided=False)
    assert torch.allclose(F1, torch.tensor([[mu * g * 0.01, 0, 0], [mu * g * 0.02, 0, 0]], dtype=DT),
                          atol=1e-12)
    F2 = O.probe_traction(fields, C, nrm, A, N, H, 0.3, mu, sum(H) / 3, two_sided=True)
    assert float(F2.abs().max()) < 1e-12
