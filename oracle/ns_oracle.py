"""FP64 CPU oracle of the coupled flow solver (the fluid phase of Sec. 2.1
and the coupled step of Sec. 5).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
baseline leg of the benchmark may import this module.  The CUDA library never
calls it, shares no code with it and does not fall back to it.

Plain PyTorch CPU tensor ops in float64 on the triply periodic MAC grid of
the Lagrangian oracle (u at (i, j+1/2, k+1/2) h, v at (i+1/2, j, k+1/2) h,
w at (i+1/2, j+1/2, k) h, the pressure at the cell centres
(i+1/2, j+1/2, k+1/2) h; arrays [nz, ny, nx]):

* incompressible Navier-Stokes, Eqs. ns and con, with nu = 1/Re and density 1;
* second-order centred conservative (divergence-form) differences on the
  staggered grid for the nonlinear terms, the 7-point Laplacian for the
  viscous terms (Sec. 2.1);
* the self-starting fractional-step RK3 of Sec. 2.1: explicit nonlinear
  terms with the three-substep weights gamma = (8/15, 5/12, 3/4),
  rho = (0, -17/60, -5/12), alpha = gamma + rho, Crank-Nicolson viscous terms
  with the approximate factorisation of the implicit operator into its three
  directional factors, and a pressure-correction Poisson equation;
* the coupled step of Sec. 5: per substep the provisional velocity is
  interpolated at the face centroids (MLS), the direct-forcing marker force
  is spread and corrects the provisional velocity, then the pressure
  correction makes it solenoidal (steps 3a, 3b, 3d, 3e); after the three
  substeps the bodies advance with the external loads (pressure and viscous
  traction at the probes) and the internal loads (step 4), as in the
  Lagrangian oracle.

Readings (also listed in the design notes):
  N1 RK3 weights: the three-substep scheme of the cited solver (Verzicco and
     Orlandi; Rai and Moin) that the paper names without coefficients.
  N2 the box is triply periodic (as the Lagrangian path); the factorised
     Crank-Nicolson operator (1 - a d_xx)(1 - a d_yy)(1 - a d_zz) and the
     Poisson operator are then diagonal in Fourier space, so both are solved
     there exactly (the library FFT is a step here); their eigenvalues are
     those of the second-order differences, -(4/h^2) sin^2(pi k / n).
  N3 pressure update p <- p + phi - alpha dt nu/2 lap(phi) (the correction
     that keeps the scheme second order with Crank-Nicolson viscous terms).
  N4 IBM forcing per substep: F = (V^b - U*)/dt with U* the provisional
     velocity at the centroids of x^n and V^b the centroid velocity of v^n;
     the provisional velocity becomes u* + dt f with f the spread of F
     (Eq. mls_cl); the markers stay at x^n during the three substeps.
  N5 the viscosity of the probe traction is the flow's nu (density 1).
"""
from __future__ import annotations

import torch

from . import ibm_oracle as O

DT = torch.float64

GAMMA = (8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0)
RHO = (0.0, -17.0 / 60.0, -5.0 / 12.0)
ALPHA = tuple(g + r for g, r in zip(GAMMA, RHO))

# array axes of [nz, ny, nx] fields for directions x, y, z
_AX = (2, 1, 0)


def shift(f, d, s):
    """f at index i + s along direction d (periodic): shift(f, d, 1)[i] = f[i+1]."""
    return torch.roll(f, -s, dims=_AX[d])


def laplacian(f, h):
    """7-point Laplacian of a field on any of the staggered lattices."""
    out = torch.zeros_like(f)
    for d in range(3):
        out = out + (shift(f, d, 1) - 2.0 * f + shift(f, d, -1)) / h[d] ** 2
    return out


def divergence(u, h):
    """Discrete divergence at the cell centres: sum_d (u_d[i_d + 1] - u_d[i_d]) / h_d."""
    return sum((shift(u[d], d, 1) - u[d]) / h[d] for d in range(3))


def gradient(p, h):
    """Gradient of a cell-centred field at the velocity nodes: component d at
    face i_d is (p[i_d] - p[i_d - 1]) / h_d."""
    return torch.stack([(p - shift(p, d, -1)) / h[d] for d in range(3)])


def advection(u, h):
    """H = -div(u u) in conservative form on the staggered grid (Sec. 2.1).

    Component c at its node: -(sum_d d_d (u_d u_c)), where the product is
    formed where the difference needs it:
      d = c: at the cell centres, from the mean of the two neighbouring c
             nodes, squared;
      d != c: at the edge between the two lattices, from the mean of u_d over
             the two u_d nodes along c times the mean of u_c over the two
             u_c nodes along d.
    """
    H = []
    for c in range(3):
        acc = torch.zeros_like(u[c])
        for d in range(3):
            if d == c:
                uc = 0.5 * (u[c] + shift(u[c], c, 1))        # cell centre i + 1/2
                q = uc * uc
                acc = acc + (q - shift(q, c, -1)) / h[c]
            else:
                ud = 0.5 * (u[d] + shift(u[d], c, -1))       # u_d at the (c, d) edge
                uc = 0.5 * (u[c] + shift(u[c], d, -1))       # u_c at the same edge
                q = ud * uc
                acc = acc + (shift(q, d, 1) - q) / h[d]
        H.append(-acc)
    return torch.stack(H)


def _eigen(n, h):
    """Eigenvalues of the periodic second difference per direction for the
    rfftn layout (the last axis, x, is halved)."""
    lam = []
    for d in range(3):
        m = n[d] // 2 + 1 if d == 0 else n[d]
        k = torch.arange(m, dtype=DT)
        lam.append(-(4.0 / h[d] ** 2) * torch.sin(torch.pi * k / n[d]) ** 2)
    lx, ly, lz = lam
    return lx[None, None, :], ly[None, :, None], lz[:, None, None]


def solve_poisson(rhs, n, h):
    """phi with lap(phi) = rhs - mean(rhs) and mean(phi) = 0 (reading N2)."""
    lx, ly, lz = _eigen(n, h)
    R = torch.fft.rfftn(rhs)
    lam = lx + ly + lz
    lam[0, 0, 0] = 1.0
    P = R / lam
    P[0, 0, 0] = 0.0
    return torch.fft.irfftn(P, s=rhs.shape)


def solve_factorised(rhs, a, n, h):
    """x with (1 - a d_xx)(1 - a d_yy)(1 - a d_zz) x = rhs (reading N2)."""
    lx, ly, lz = _eigen(n, h)
    R = torch.fft.rfftn(rhs)
    X = R / ((1.0 - a * lx) * (1.0 - a * ly) * (1.0 - a * lz))
    return torch.fft.irfftn(X, s=rhs.shape)


class Flow:
    """Grid, viscosity and time step of the fluid phase."""

    def __init__(self, n, L=(1.0, 1.0, 1.0), nu=1.0, dt=1e-3):
        self.n = tuple(int(v) for v in n)
        self.L = tuple(float(v) for v in L)
        self.h = tuple(self.L[d] / self.n[d] for d in range(3))
        self.nu, self.dt = float(nu), float(dt)


def predict(flow: Flow, l, u, p, H_prev):
    """Provisional velocity of RK3 substep l (0, 1, 2), Sec. 2.1:
      (u* - u)/dt = gamma_l H(u) + rho_l H_prev - alpha_l grad p
                    + alpha_l nu/2 lap(u* + u),
    with the implicit operator approximately factorised (reading N2).
    Returns (u*, H(u))."""
    h, dt, nu = flow.h, flow.dt, flow.nu
    H = advection(u, h)
    G = gradient(p, h)
    a = ALPHA[l] * dt * nu / 2.0
    out = []
    for c in range(3):
        rhs = GAMMA[l] * H[c] - ALPHA[l] * G[c] + ALPHA[l] * nu * laplacian(u[c], h)
        if RHO[l] != 0.0:
            rhs = rhs + RHO[l] * H_prev[c]
        out.append(u[c] + solve_factorised(dt * rhs, a, flow.n, h))
    return torch.stack(out), H


def project(flow: Flow, l, u_star, p):
    """Pressure correction of substep l: lap(phi) = div(u*)/(alpha_l dt),
    u = u* - alpha_l dt grad(phi), p <- p + phi - alpha_l dt nu/2 lap(phi)
    (reading N3).  Returns (u, p)."""
    h, dt, nu = flow.h, flow.dt, flow.nu
    phi = solve_poisson(divergence(u_star, h) / (ALPHA[l] * dt), flow.n, h)
    u = u_star - ALPHA[l] * dt * gradient(phi, h)
    p = p + phi - ALPHA[l] * dt * nu / 2.0 * laplacian(phi, h)
    return u, p


def ns_step(flow: Flow, u, p):
    """One time step of the flow alone (three substeps)."""
    H_prev = None
    for l in range(3):
        u_star, H_prev = predict(flow, l, u, p, H_prev)
        u, p = project(flow, l, u_star, p)
    return u, p


def ibm_forcing(bodies, xs, vs, u_star, prm: O.Params):
    """Spread direct-forcing field of one substep (reading N4): F = (V^b - U*)/dt
    at the centroids of xs, f = spread(F) (Eq. mls_cl).  Returns f [3,nz,ny,nx]."""
    n, h, alpha, dt = prm.n, prm.h, prm.alpha, prm.dt
    Cs, As, Fs = [], [], []
    for b, x, v in zip(bodies, xs, vs):
        C, _, A_l = O.face_geometry(x, b.tri)
        Vb = (v[b.tri[:, 0]] + v[b.tri[:, 1]] + v[b.tri[:, 2]]) / 3.0
        U = torch.stack([O.interpolate(u_star[i], C, i, n, h, alpha) for i in range(3)], 1)
        Cs.append(C)
        As.append(A_l)
        Fs.append((Vb - U) / dt)
    return O.spread(torch.cat(Fs), torch.cat(Cs), torch.cat(As), n, h, alpha)


def coupled_step(bodies, xs, vs, u, p, flow: Flow, prm: O.Params):
    """One loosely coupled time step (Sec. 5 steps 1-4): three RK3 substeps of
    the flow, each with the IBM correction of the provisional velocity before
    the pressure correction, then the body update with the loads of the new
    flow (pressure and viscous traction; F_int) by the Lagrangian oracle.
    prm carries the MLS and body parameters (its mu is the flow's nu, its dt
    the flow's dt).  Returns (x_next, v_next, u, p, f of the last substep)."""
    f = torch.zeros_like(u)
    H_prev = None
    for l in range(3):
        u_star, H_prev = predict(flow, l, u, p, H_prev)           # 3a
        if bodies:
            f = ibm_forcing(bodies, xs, vs, u_star, prm)          # 3b
            u_star = u_star + prm.dt * f                          # 3d
        u, p = project(flow, l, u_star, p)                        # 3e
    if bodies:
        out = O.step(bodies, xs, vs, tuple(u), prm, with_spread=False, pressure=p)   # 4
        xs, vs = out["x_next"], out["v_next"]
    return xs, vs, u, p, f
