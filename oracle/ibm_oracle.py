"""FP64 CPU oracle of the Lagrangian interaction-potential + MLS-IBM step.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
baseline leg of the benchmark may import this module.  The CUDA library never
calls it, shares no code with it and does not fall back to it.

It is a plain, slow, literal restatement of the method of Spandan et al.,
"A parallel interaction potential approach coupled with the immersed boundary
method for fully resolved simulations of deformable interfaces and membranes"
(J. Comp. Phys.), written with plain PyTorch CPU tensor ops in float64:

* geometry of the triangulated surface, centroids as Lagrangian markers
  (Sec. 2.2, Fig. lagmesh);
* the four interaction potentials W_e, W_b, W_v, W_a (Sec. 2.3, Eqs.
  elaspot..areapot); nodal forces are their exact negative gradients, taken
  here by automatic differentiation of the energy (the "spatial derivative
  operation" of Sec. 2.3);
* the MLS transfer function with linear basis, exponential weight and a
  3x3x3 support (Sec. 2.2, Eqs. mls..mls_Q), solved as a general 4x4 system
  by LU with partial pivoting, and its full derivative for the probe
  gradient (Sec. 5.1);
* the direct-forcing marker force F = (V^b - U)/dt and its spreading with the
  c_l scaling (Sec. 2.2, Eq. mls_cl);
* the probe traction F_ext = (-p n + tau . n) A (one-sided probe for closed
  bodies, two-sided for open sheets) and the 1/3 face-to-vertex distribution
  (Sec. 2.2, Sec. 2.3);
* the node update m x'' = F_ext + F_int (Sec. 2.3, Sec. 5 step 4).

Readings of passages the paper leaves open (each one is listed, with its
reason, in the design notes of the repository):
  R1 Eq. mls_A: A = sum_k W_k p(x^k) p(x^k)^T (the printed p(x) p^T(x^k) is
     read as the standard MLS moment matrix, consistent with Eq. mls_B).
  R2 Eq. mls_cl / the spreading formula: the sum runs over the markers l
     whose support holds node k; Delta V^K is the cell volume at node k.
  R3 Eqs. mls_w, mls_rk: r_k^2 = sum_d ((x_d - x_d^k) / r_d)^2 with
     r_d = 1.5 h_d; every one of the 27 nodes is within r_d per direction, so
     all 27 are kept; W = exp(-r_k^2 / alpha^2).
  R4 alpha (not given): 0.3 by default, a parameter.
  R5 staggering: MAC lattice, u at (i, j+1/2, k+1/2) h, v at
     (i+1/2, j, k+1/2) h, w at (i+1/2, j+1/2, k) h; the stencil centre is the
     nearest node floor(t + 1/2) of that component's lattice; indices wrap
     (triply periodic box).
  R6 W_b: theta is the signed angle between the two face normals,
     cos = n1.n2, sin = (n1 x n2).e; W_b = k_b (1 - cos(theta - theta0)) with
     theta0 the rest angle (theta0 = 0 is the literal text, a flag).
  R7 W_a: a local term per face with its own A0_f plus a global per-body term;
     W_v is per closed body (divergence theorem); k_v = 0 on open sheets.
  R8 integrator: symplectic Euler with F_int at x^n, which is the paper's
     "internal force of the previous time step"; v^0 = 0.  Forward Euler is a
     flag.
  R9 x in W_e is l - l0 with l0 the rest length; k_e = k_s uniform.
  R10 frozen flow: p = 0 unless a pressure field is supplied, viscosity mu
     (1), probe length h = mean grid spacing.
  R11 the probe gradient uses the full derivative of the shape function.
  R12 node mass m per body (1 for drops).
  R16 pressure (when supplied) lives at the cell centres, (i+1/2, j+1/2,
     k+1/2) h; the marker acceleration Du/Dt of the correction
     p_l = p* + h (Du/Dt).n is the mean of the face's three vertex
     accelerations, which the caller supplies (e.g. (v^n - v^(n-1))/dt).
  R17 open sheets: each side takes p^+- = p*^+- + h (Du/Dt).n^+- with
     n^+- = +-n^+, and the load is -(p^+ - p^-) n^+ A.
  R18 non-uniform meshes and materials: k_e per edge by van Gelder's model,
     k_e = k_s sum over the edge's faces of A_T / l_e^2 (rest values; k_s is
     then the membrane's E t); per-face material multipliers of (k_s, k_b,
     k_a): an edge takes the mean of its faces' (the area-weighted sum under
     van Gelder), a hinge the mean of its two faces', a face its own.
  R19 strong coupling (Sec. 2.3) with the flow frozen: the fluid-structure
     iteration reduces to Hamming's fourth-order predictor-corrector for
     y = (x, v), y' = (v, (F_int + F_ext^v)/m), one corrector application per
     step as in the classical scheme, started by three classical Runge-Kutta
     steps.
"""
from __future__ import annotations

import math

import torch

DT = torch.float64

MAC_OFFSET = ((0.0, 0.5, 0.5), (0.5, 0.0, 0.5), (0.5, 0.5, 0.0), (0.5, 0.5, 0.5))
"""Offsets in cells of the u, v, w node lattices (reading R5) and of the
cell-centred pressure lattice (index 3, reading R16)."""


# --------------------------------------------------------------------------
# topology (Sec. 5: vert_of_edge, face_of_edge, v1234 ...)
# --------------------------------------------------------------------------


class MeshError(ValueError):
    pass


def build_topology(tri, n_vert):
    """Edges and hinges of an oriented triangle mesh (Sec. 5, the
    vert_of_edge / face_of_edge / v1234 arrays).

    Returns a dict with
      edges  [E,2]: (a, b), oriented as in the first face that holds it;
      wings  [E,2]: (c, d): c the third vertex of the face holding a->b,
                    d the third vertex of the face holding b->a, -1 if none;
      efaces [E,2]: those two faces (-1 if none).
    Raises MeshError on an edge shared by more than two faces or by two
    faces with the same direction (inconsistent orientation).
    """
    tri = [tuple(int(v) for v in t) for t in tri]
    half = {}
    for f, (a, b, c) in enumerate(tri):
        if len({a, b, c}) != 3:
            raise MeshError(f"degenerate face {f}")
        for p, q, r in ((a, b, c), (b, c, a), (c, a, b)):
            if not (0 <= p < n_vert):
                raise MeshError(f"vertex index out of range in face {f}")
            if (p, q) in half:
                raise MeshError(f"edge ({p},{q}) used twice in the same direction")
            half[(p, q)] = (f, r)
    edges, wings, efaces, seen = [], [], [], set()
    for f, (a, b, c) in enumerate(tri):
        for p, q, r in ((a, b, c), (b, c, a), (c, a, b)):
            key = (min(p, q), max(p, q))
            if key in seen:
                continue
            seen.add(key)
            f2, s = half.get((q, p), (-1, -1))
            edges.append((p, q))
            wings.append((r, s))
            efaces.append((f, f2))
    t = lambda a: torch.tensor(a, dtype=torch.long).reshape(-1, 2)
    return {"edges": t(edges), "wings": t(wings), "efaces": t(efaces),
            "tri": torch.tensor(tri, dtype=torch.long).reshape(-1, 3)}


# --------------------------------------------------------------------------
# surface geometry (Sec. 2.2)
# --------------------------------------------------------------------------


def face_geometry(x, tri):
    """Per face: centroid (the Lagrangian marker, mean of the three vertices
    since mass is uniform on the face), unit normal, area."""
    xa, xb, xc = x[tri[:, 0]], x[tri[:, 1]], x[tri[:, 2]]
    N = torch.cross(xb - xa, xc - xa, dim=1)
    nrm = torch.linalg.vector_norm(N, dim=1)
    return (xa + xb + xc) / 3.0, N / nrm[:, None], 0.5 * nrm


def edge_lengths(x, edges):
    return torch.linalg.vector_norm(x[edges[:, 1]] - x[edges[:, 0]], dim=1)


def hinge_angle(x, edges, wings):
    """cos and sin of the signed angle between the normals of the two faces
    of each interior edge (reading R6).  Face 1 = (a, b, c), face 2 =
    (b, a, d); sin = (n1 x n2) . e_ab, positive for a convex ridge."""
    a, b, c, d = edges[:, 0], edges[:, 1], wings[:, 0], wings[:, 1]
    xa, xb, xc, xd = x[a], x[b], x[c], x[d]
    n1 = torch.cross(xb - xa, xc - xa, dim=1)
    n2 = torch.cross(xa - xb, xd - xb, dim=1)
    n1 = n1 / torch.linalg.vector_norm(n1, dim=1, keepdim=True)
    n2 = n2 / torch.linalg.vector_norm(n2, dim=1, keepdim=True)
    e = xb - xa
    e = e / torch.linalg.vector_norm(e, dim=1, keepdim=True)
    cos = (n1 * n2).sum(1)
    sin = (torch.cross(n1, n2, dim=1) * e).sum(1)
    return cos, sin


def enclosed_volume(x, tri, origin):
    """Volume of a closed oriented surface, sum of signed tetrahedra
    (origin, a, b, c) (divergence theorem)."""
    y = x - origin
    return (y[tri[:, 0]] * torch.cross(y[tri[:, 1]], y[tri[:, 2]], dim=1)).sum() / 6.0


# --------------------------------------------------------------------------
# bodies and the interaction potentials (Sec. 2.3)
# --------------------------------------------------------------------------


class Body:
    """One triangulated body with its rest state and elastic constants.

    rest: [V,3] absolute rest positions (float64); tri: [F,3] outward CCW;
    origin: [3] body-frame origin (a point near the body centre, used only to
    keep volume sums well conditioned).  Constants k_s, k_b, k_a (local
    area), k_A (global area), k_v (volume) and the node mass are float64
    tensors so that gradients can be taken with respect to them.
    """

    def __init__(self, rest, tri, origin, closed=True, clamped=None, ks=1.0, kb=0.01,
                 ka=1.0, kA=1.0, kv=1.0, mass=1.0, theta0_zero=False, spring_model=0,
                 face_material=None):
        self.rest = torch.as_tensor(rest, dtype=DT)
        self.nv = self.rest.shape[0]
        self.topo = build_topology(tri, self.nv)
        self.tri = self.topo["tri"]
        self.origin = torch.as_tensor(origin, dtype=DT)
        self.closed = bool(closed)
        self.clamped = (torch.zeros(self.nv, dtype=torch.bool) if clamped is None
                        else torch.as_tensor(clamped, dtype=torch.bool))
        kt = lambda v: torch.as_tensor(float(v), dtype=DT)
        self.ks, self.kb, self.ka, self.kA = kt(ks), kt(kb), kt(ka), kt(kA)
        self.kv = kt(kv if closed else 0.0)
        self.mass = kt(mass)
        inner = self.topo["wings"][:, 1] >= 0
        self.hinge_edges = self.topo["edges"][inner]
        self.hinge_wings = self.topo["wings"][inner]
        if self.closed and not bool(inner.all()):
            raise MeshError("closed body has boundary edges")
        # rest state: l0, theta0 (as cos/sin), A0_f, A0, V0
        with torch.no_grad():
            self.l0 = edge_lengths(self.rest, self.topo["edges"])
            c0, s0 = hinge_angle(self.rest, self.hinge_edges, self.hinge_wings)
            if theta0_zero:
                c0, s0 = torch.ones_like(c0), torch.zeros_like(s0)
            self.cos0, self.sin0 = c0, s0
            _, _, A0f = face_geometry(self.rest, self.tri)
            self.A0f = A0f
            self.A0 = A0f.sum()
            self.V0 = enclosed_volume(self.rest, self.tri, self.origin) if closed else torch.tensor(0.0, dtype=DT)
            if closed and self.V0 <= 0:
                raise MeshError("closed body has non-positive rest volume (inward faces?)")
            self._element_scales(spring_model, face_material)

    def _element_scales(self, spring_model, face_material):
        """Per-element multipliers of k_s (edges), k_b (hinges) and k_a (faces)
        (reading R18).  face_material [F,3]: per-face (m_s, m_b, m_a), ones if
        None.  Spring model 0: m_e = mean of m_s over the edge's faces;
        model 1 (van Gelder): m_e = sum over the edge's faces T of
        m_s(T) A_T / l_e^2 (rest areas and lengths), so that k_s is the
        membrane's E t.  A hinge takes the mean m_b of its two faces."""
        F = self.tri.shape[0]
        m = (torch.ones(F, 3, dtype=DT) if face_material is None
             else torch.as_tensor(face_material, dtype=DT).reshape(F, 3))
        ef = self.topo["efaces"]
        has2 = ef[:, 1] >= 0
        f0, f1 = ef[:, 0], ef[:, 1].clamp(min=0)
        ms0, ms1 = m[f0, 0], torch.where(has2, m[f1, 0], torch.zeros_like(m[f0, 0]))
        if spring_model == 0:
            self.m_edge = (ms0 + ms1) / torch.where(has2, 2.0, 1.0).to(DT)
        elif spring_model == 1:
            A0 = self.A0f
            area = ms0 * A0[f0] + torch.where(has2, ms1 * A0[f1], torch.zeros_like(ms1))
            self.m_edge = area / self.l0 ** 2
        else:
            raise ValueError("spring_model must be 0 or 1")
        inner = ef[:, 1] >= 0
        self.m_hinge = 0.5 * (m[ef[inner, 0], 1] + m[ef[inner, 1], 1])
        self.m_face = m[:, 2].clone()

    def energy_terms(self, x):
        """W_e, W_b, W_a (local), W_A (global), W_v of Sec. 2.3 at positions x."""
        l = edge_lengths(x, self.topo["edges"])
        We = 0.5 * self.ks * (self.m_edge * (l - self.l0) ** 2).sum()         # Eq. elaspot
        cos, sin = hinge_angle(x, self.hinge_edges, self.hinge_wings)
        Wb = (self.kb * self.m_hinge * (1.0 - (cos * self.cos0 + sin * self.sin0))).sum()
        _, _, Af = face_geometry(x, self.tri)
        Wa = (0.5 * self.ka * self.m_face * (Af - self.A0f) ** 2 / self.A0f).sum()   # Eq. areapot
        A = Af.sum()
        WA = 0.5 * self.kA * (A - self.A0) ** 2 / self.A0                     # Eq. areapot, per body
        if self.closed:
            V = enclosed_volume(x, self.tri, self.origin)
            Wv = 0.5 * self.kv * (V - self.V0) ** 2 / self.V0                 # volume potential
        else:
            Wv = torch.zeros((), dtype=DT)
        return {"We": We, "Wb": Wb, "Wa": Wa, "WA": WA, "Wv": Wv}

    def energy(self, x):
        t = self.energy_terms(x)
        return t["We"] + t["Wb"] + t["Wa"] + t["WA"] + t["Wv"]

    def internal_forces(self, x, create_graph=False):
        """F_int = -dW/dx (Sec. 2.3: nodal forces from the potentials by a
        spatial derivative), exact, by reverse-mode differentiation."""
        xx = x if x.requires_grad else x.detach().requires_grad_(True)
        W = self.energy(xx)
        (g,) = torch.autograd.grad(W, xx, create_graph=create_graph)
        return -g


# --------------------------------------------------------------------------
# MLS transfer function (Sec. 2.2, Eqs. mls..mls_Q)
# --------------------------------------------------------------------------

_S = torch.tensor([(sx, sy, sz) for sz in (-1, 0, 1) for sy in (-1, 0, 1) for sx in (-1, 0, 1)],
                  dtype=DT)           # stencil offsets, x fastest


def mls_stencil(P, comp, n, h):
    """27-node support of each point for velocity component `comp`: the
    nearest node of that component's lattice and its +-1 neighbours
    (reading R5).  Returns (flat indices [M,27] into an [nz,ny,nx] array,
    node positions [M,27,3] unwrapped around P, centre node [M,3])."""
    off = torch.tensor(MAC_OFFSET[comp], dtype=DT)
    hh = torch.tensor(h, dtype=DT)
    t = P.detach() / hh - off
    ic = torch.floor(t + 0.5)
    nodes = ic[:, None, :] + _S[None]                  # lattice coords
    pos = (nodes + off) * hh
    nn = torch.tensor(n, dtype=torch.long)
    w = torch.remainder(nodes.long(), nn)
    flat = (w[..., 2] * n[1] + w[..., 1]) * n[0] + w[..., 0]
    return flat, pos, (ic + off) * hh


def mls_weight(P, pos, h, alpha):
    """Exponential weight W = exp(-(r_k/alpha)^2) with the per-direction
    normalised distance of reading R3 (Eqs. mls_w, mls_rk)."""
    r = torch.tensor([1.5 * hd for hd in h], dtype=DT)
    q = (pos - P[:, None, :]) / r
    return torch.exp(-(q * q).sum(-1) / alpha ** 2)


def mls_shape(P, comp, n, h, alpha, with_grad=False):
    """MLS shape functions phi^T = p^T(x) A^{-1} B at points P (Eq. mls_Q),
    with A = sum_k W_k p(x^k) p(x^k)^T (reading R1, Eq. mls_A),
    B = [W_k p(x^k)] (Eq. mls_B), linear basis p = [1, x, y, z] (Eq. mls)
    expressed about the stencil centre node.  The 4x4 systems are solved by
    LU with partial pivoting.

    with_grad: also the full derivative d phi / d x (reading R11):
      dphi = dp^T A^-1 B - p^T A^-1 dA A^-1 B + p^T A^-1 dB.
    Returns (flat [M,27], phi [M,27]) or (flat, phi, dphi [M,27,3]).
    """
    flat, pos, centre = mls_stencil(P, comp, n, h)
    W = mls_weight(P, pos, h, alpha)                                  # [M,27]
    M = P.shape[0]
    pk = torch.cat([torch.ones(M, 27, 1, dtype=DT), pos - centre[:, None, :]], -1)   # [M,27,4]
    px = torch.cat([torch.ones(M, 1, dtype=DT), P - centre], -1)                     # [M,4]
    A = torch.einsum("mk,mki,mkj->mij", W, pk, pk)
    B = (W[..., None] * pk).transpose(1, 2)                                            # [M,4,27]
    G = torch.linalg.solve(A, B)                                                       # A^-1 B
    phi = torch.einsum("mi,mik->mk", px, G)
    if not with_grad:
        return flat, phi
    r2 = torch.tensor([(1.5 * hd) ** 2 for hd in h], dtype=DT)
    delta = pos - P[:, None, :]
    dW = W[..., None] * (2.0 / alpha ** 2) * delta / r2                               # dW_k/dx_e
    rvec = torch.linalg.solve(A, px[..., None])[..., 0]                                # A^-1 p (A symmetric)
    dphi = []
    for e in range(3):
        dA = torch.einsum("mk,mki,mkj->mij", dW[..., e], pk, pk)
        dB = (dW[..., e][..., None] * pk).transpose(1, 2)
        term1 = G[:, e + 1, :]
        term2 = -torch.einsum("mi,mij,mjk->mk", rvec, dA, G)
        term3 = torch.einsum("mi,mik->mk", rvec, dB)
        dphi.append(term1 + term2 + term3)
    return flat, phi, torch.stack(dphi, -1)


def interpolate(field, P, comp, n, h, alpha):
    """U(P) = sum_k phi_k q^k (Eq. mls_Q) for one velocity component."""
    flat, phi = mls_shape(P, comp, n, h, alpha)
    return (phi * field.reshape(-1)[flat]).sum(1)


def interpolate_gradient(field, P, comp, n, h, alpha):
    """grad U(P) = sum_k dphi_k q^k (full derivative, Sec. 5.1)."""
    flat, phi, dphi = mls_shape(P, comp, n, h, alpha, with_grad=True)
    q = field.reshape(-1)[flat]
    return (dphi * q[..., None]).sum(1)


# --------------------------------------------------------------------------
# IBM forcing and spreading (Sec. 2.2)
# --------------------------------------------------------------------------


def spread(F, P, A_l, n, h, alpha, out=None):
    """Spread marker forces F [M,3] to the three staggered force fields:
    f_i^k += c_l phi_k^l F_i^l with c_l = dV^l / sum_k phi_k^l dV^k,
    dV^l = A_l h_l, h_l = 1/3 sum_k phi_k^l (dx^k + dy^k + dz^k)
    (Eq. mls_cl; reading R2).  Returns [3, nz, ny, nx]."""
    nx, ny, nz = n
    dVk = h[0] * h[1] * h[2]
    hsum = h[0] + h[1] + h[2]
    fields = []
    for comp in range(3):
        flat, phi = mls_shape(P, comp, n, h, alpha)
        h_l = (phi * hsum).sum(1) / 3.0
        dVl = A_l * h_l
        c_l = dVl / (phi * dVk).sum(1)
        contrib = (c_l[:, None] * phi * F[:, comp:comp + 1]).reshape(-1)
        f = torch.zeros(nx * ny * nz, dtype=DT)
        f = f.index_add(0, flat.reshape(-1), contrib)
        if out is not None:
            f = f + out[comp].reshape(-1)
        fields.append(f.reshape(nz, ny, nx))
    return torch.stack(fields)


def probe_traction(fields, C, nrm, A_l, n, h, alpha, mu, probe_h, two_sided, pressure=None,
                   accel=None):
    """External load per face, F_ext = (-p n + tau . n) A (Sec. 2.2), with
    tau = mu (grad u + grad u^T) from the MLS gradient at the probe end
    c + h n, and p = 0 (frozen flow, reading R10) or, with a pressure field,
    p = p* + h (Du/Dt).n with p* interpolated at the probe end and Du/Dt the
    marker acceleration accel [M,3] (zero if None; reading R16).  Two-sided
    for open sheets: F_ext = (-(p+ - p-) n+ + (tau+ - tau-) . n+) A, each side
    with its own normal +-n+ (reading R17)."""

    def tau_dot_n(Pp):
        G = torch.stack([interpolate_gradient(fields[i], Pp, i, n, h, alpha) for i in range(3)], 1)
        tau = mu * (G + G.transpose(1, 2))                       # [M,3,3], G[i,j] = du_i/dx_j
        return torch.einsum("mij,mj->mi", tau, nrm)

    def marker_pressure(side):
        ns = side * nrm
        p_star = interpolate(pressure, C + probe_h * ns, 3, n, h, alpha)
        if accel is None:
            return p_star
        return p_star + probe_h * (accel * ns).sum(1)

    F = tau_dot_n(C + probe_h * nrm)
    if two_sided:
        F = F - tau_dot_n(C - probe_h * nrm)
    if pressure is not None:
        p = marker_pressure(1.0)
        if two_sided:
            p = p - marker_pressure(-1.0)
        F = F - p[:, None] * nrm
    return F * A_l[:, None]


def distribute_to_vertices(Fface, tri, nv):
    """F_ext^v = sum over the faces j holding v of F_ext^{c_j} / 3 (Sec. 2.3)."""
    out = torch.zeros(nv, 3, dtype=DT)
    for k in range(3):
        out = out.index_add(0, tri[:, k], Fface / 3.0)
    return out


def advance(b, x, v, F_int, F_ext_face, prm):
    """Node update of one body (Sec. 2.3, m x'' = F_ext + F_int; Sec. 5 step
    4): the face loads are distributed a third to each corner, then
    symplectic Euler (reading R8: v' = v + dt a, x' = x + dt v') or forward
    Euler (x' = x + dt v, v' = v + dt a); clamped nodes keep x and get v = 0.
    Returns (x', v', F_ext per vertex)."""
    dt = prm.dt
    Fev = distribute_to_vertices(F_ext_face, b.tri, b.nv)
    acc = (Fev + F_int) / b.mass
    if prm.forward_euler:
        xn = x + dt * v
        vn = v + dt * acc
    else:
        vn = v + dt * acc
        xn = x + dt * vn
    cl = b.clamped[:, None]
    xn = torch.where(cl, x, xn)
    vn = torch.where(cl, torch.zeros_like(vn), vn)
    return xn, vn, Fev


# --------------------------------------------------------------------------
# one loosely coupled step (Sec. 5 steps 1, 2, 3b, 4) with the flow frozen
# --------------------------------------------------------------------------


class Params:
    def __init__(self, n, L=(1.0, 1.0, 1.0), dt=1e-3, mu=1.0, alpha=0.3, probe_h=None,
                 forward_euler=False):
        self.n = tuple(int(v) for v in n)
        self.L = tuple(float(v) for v in L)
        self.h = tuple(self.L[d] / self.n[d] for d in range(3))
        self.dt, self.mu, self.alpha = float(dt), float(mu), float(alpha)
        self.probe_h = float(probe_h) if probe_h is not None else sum(self.h) / 3.0
        self.forward_euler = bool(forward_euler)


def step(bodies, xs, vs, fields, prm: Params, create_graph=False, with_spread=True,
         pressure=None, accels=None):
    """One step for every body.  xs, vs: lists of [V,3] absolute positions
    and velocities; fields: (u, v, w) [nz,ny,nx] float64; pressure: None or
    the cell-centred pressure [nz,ny,nx]; accels: None or a list of [V,3]
    vertex accelerations (the marker acceleration is their face mean).
    Returns a dict with x_next, v_next (lists), F_int, F_ext_vertex (lists),
    and per-marker U, F_marker, F_ext_face, plus the spread force fields
    f [3,nz,ny,nx]."""
    n, h, alpha, dt = prm.n, prm.h, prm.alpha, prm.dt
    x_next, v_next, Fint_l, Fextv_l = [], [], [], []
    Us, Fms, Fes, Ps, As = [], [], [], [], []
    for ib, (b, x, v) in enumerate(zip(bodies, xs, vs)):
        C, nrm, A_l = face_geometry(x, b.tri)                                # steps 1, 2
        acc_l = None
        if pressure is not None and accels is not None:
            a = accels[ib]
            acc_l = (a[b.tri[:, 0]] + a[b.tri[:, 1]] + a[b.tri[:, 2]]) / 3.0
        Vb = (v[b.tri[:, 0]] + v[b.tri[:, 1]] + v[b.tri[:, 2]]) / 3.0       # marker velocity
        U = torch.stack([interpolate(fields[i], C, i, n, h, alpha) for i in range(3)], 1)   # 3b
        Fm = (Vb - U) / dt                                                   # F = (V^b - U)/dt
        Fe = probe_traction(fields, C, nrm, A_l, n, h, alpha, prm.mu, prm.probe_h,
                            two_sided=not b.closed, pressure=pressure, accel=acc_l)   # 4a
        Fi = b.internal_forces(x, create_graph=create_graph)                # 4c
        xn, vn, Fev = advance(b, x, v, Fi, Fe, prm)                         # 4d, 4e
        x_next.append(xn)
        v_next.append(vn)
        Fint_l.append(Fi)
        Fextv_l.append(Fev)
        Us.append(U)
        Fms.append(Fm)
        Fes.append(Fe)
        Ps.append(C)
        As.append(A_l)
    out = {"x_next": x_next, "v_next": v_next, "F_int": Fint_l, "F_ext_vertex": Fextv_l,
           "U": torch.cat(Us), "F_marker": torch.cat(Fms), "F_ext_face": torch.cat(Fes),
           "markers": torch.cat(Ps), "areas": torch.cat(As)}
    if with_spread:
        out["f"] = spread(out["F_marker"], out["markers"], out["areas"], n, h, alpha)
    return out


# --------------------------------------------------------------------------
# strong coupling: Hamming's fourth-order predictor-corrector (Sec. 2.3)
# --------------------------------------------------------------------------


def accelerations(bodies, xs, fields, prm: Params, pressure=None, accels=None):
    """a = (F_int + F_ext^v)/m per vertex at positions xs (the right-hand side
    of m x'' = F_ext + F_int, Sec. 2.3); clamped nodes get a = 0."""
    n, h, alpha = prm.n, prm.h, prm.alpha
    out = []
    for ib, (b, x) in enumerate(zip(bodies, xs)):
        C, nrm, A_l = face_geometry(x, b.tri)
        acc_l = None
        if pressure is not None and accels is not None:
            a = accels[ib]
            acc_l = (a[b.tri[:, 0]] + a[b.tri[:, 1]] + a[b.tri[:, 2]]) / 3.0
        Fe = probe_traction(fields, C, nrm, A_l, n, h, alpha, prm.mu, prm.probe_h,
                            two_sided=not b.closed, pressure=pressure, accel=acc_l)
        acc = (distribute_to_vertices(Fe, b.tri, b.nv) + b.internal_forces(x)) / b.mass
        out.append(torch.where(b.clamped[:, None], torch.zeros_like(acc), acc))
    return out


def rk4_step(f, y, dt):
    """One classical fourth-order Runge-Kutta step of y' = f(y)."""
    k1 = f(y)
    k2 = f(y + 0.5 * dt * k1)
    k3 = f(y + 0.5 * dt * k2)
    k4 = f(y + dt * k3)
    return y + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


class Hamming:
    """Hamming's fourth-order predictor-corrector for y' = f(y) (reading
    R19), started by three classical Runge-Kutta steps:
      predictor  p = y_{n-3} + 4h/3 (2 f_n - f_{n-1} + 2 f_{n-2})      (Milne)
      modifier   m = p - 112/121 (p_n - c_n)
      corrector  c = (9 y_n - y_{n-2})/8 + 3h/8 (f(m) + 2 f_n - f_{n-1})
      final      y_{n+1} = c + 9/121 (p - c)
    with p_n - c_n = 0 on the first Hamming step.  Each Hamming step
    evaluates f twice (at y_n and at m)."""

    def __init__(self, f, y0, dt):
        self.f, self.dt = f, dt
        self.ys = [y0]            # y_0 .. y_n (the last four are kept)
        self.fs = []              # f(y_k) for the kept y_k
        self.pc = None            # p_n - c_n

    def step(self):
        h, f = self.dt, self.f
        if len(self.ys) < 4:                      # start-up
            self.ys.append(rk4_step(f, self.ys[-1], h))
            return self.ys[-1]
        y = self.ys
        while len(self.fs) < len(y):
            self.fs.append(f(y[len(self.fs)]))
        fn, fn1, fn2 = self.fs[-1], self.fs[-2], self.fs[-3]
        p = y[-4] + (4.0 * h / 3.0) * (2.0 * fn - fn1 + 2.0 * fn2)
        m = p if self.pc is None else p - (112.0 / 121.0) * self.pc
        c = (9.0 * y[-1] - y[-3]) / 8.0 + (3.0 * h / 8.0) * (f(m) + 2.0 * fn - fn1)
        yn = c + (9.0 / 121.0) * (p - c)
        self.pc = p - c
        self.ys = self.ys[-3:] + [yn]
        self.fs = self.fs[-3:]
        return yn


def hamming_rollout(bodies, xs, vs, fields, prm: Params, n_steps, pressure=None, accels=None):
    """n_steps of the Hamming predictor-corrector (three RK4 start-up steps)
    for every body at once; y = (x, v), f(y) = (v, a(x)).  Returns the lists
    of positions and velocities after each step."""
    sizes = [len(x) for x in xs]

    def pack(xl, vl):
        return torch.stack([torch.cat(xl), torch.cat(vl)])

    def unpack(y):
        return list(torch.split(y[0], sizes)), list(torch.split(y[1], sizes))

    def f(y):
        xl, vl = unpack(y)
        al = accelerations(bodies, xl, fields, prm, pressure, accels)
        return torch.stack([y[1], torch.cat(al)])

    H = Hamming(f, pack(xs, vs), prm.dt)
    out = []
    for _ in range(n_steps):
        out.append(unpack(H.step()))
    return out


# --------------------------------------------------------------------------
# Taylor deformation of a closed body (drop semi-axes L, B of Sec. 3.1)
# --------------------------------------------------------------------------


def second_moment(x, tri, origin):
    """Volume and second-moment tensor about the centroid of the solid
    bounded by a closed oriented surface, by signed tetrahedra from `origin`
    (tetrahedron (0, p1, p2, p3): int y y^T dV = V/20 (sum p p^T + s s^T),
    s = p1 + p2 + p3)."""
    y = x - origin
    p1, p2, p3 = y[tri[:, 0]], y[tri[:, 1]], y[tri[:, 2]]
    Vt = (p1 * torch.cross(p2, p3, dim=1)).sum(1) / 6.0
    s = p1 + p2 + p3
    m1 = (Vt[:, None] * s / 4.0).sum(0)
    outer = lambda a: a[:, :, None] * a[:, None, :]
    m2 = (Vt[:, None, None] / 20.0 * (outer(p1) + outer(p2) + outer(p3) + outer(s))).sum(0)
    V = Vt.sum()
    ybar = m1 / V
    return V, m2 / V - torch.outer(ybar, ybar)


def taylor_deformation(x, tri, origin):
    """D = (L - B)/(L + B) with L, B the largest and smallest semi-axes of the
    ellipsoid with the same second moments, a_i = sqrt(5 lambda_i)."""
    _, M = second_moment(x, tri, origin)
    lam = torch.linalg.eigvalsh(M)
    a = torch.sqrt(5.0 * lam)
    return (a[-1] - a[0]) / (a[-1] + a[0])
