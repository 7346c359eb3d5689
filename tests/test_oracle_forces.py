"""Pins of the oracle's interaction-potential forces (Sec. 2.3) against
closed forms, symmetries and finite differences; no GPU."""
import math
import os

import numpy as np
import pytest
import torch

from oracle import ibm_oracle as O
from paper_1612_03399_gb300 import workloads as W

DT = torch.float64


def tetra(R=1.0):
    """Regular tetrahedron of circumradius R about the origin, outward faces."""
    p = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
    p *= R / math.sqrt(3.0)
    tri = np.array([[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]], dtype=np.int32)
    return p, tri


def only(ks=0.0, kb=0.0, ka=0.0, kA=0.0, kv=0.0):
    return dict(ks=ks, kb=kb, ka=ka, kA=kA, kv=kv)


def test_tetra_orientation_and_volume():
    p, tri = tetra(1.0)
    b = O.Body(p, tri, np.zeros(3), **only(kv=1.0))
    l0 = 2.0 * math.sqrt(2.0 / 3.0)
    assert float(b.V0) == pytest.approx(l0 ** 3 / (6.0 * math.sqrt(2.0)), rel=1e-14)
    assert float(b.A0) == pytest.approx(math.sqrt(3.0) * l0 ** 2, rel=1e-14)
    assert torch.allclose(b.l0, torch.full_like(b.l0, l0), rtol=1e-14, atol=0)


def test_mesh_counts_match_paper():
    """Icosphere sizes printed in the paper (tests/golden/paper_mesh_counts.txt)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_mesh_counts.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for level, nv, nf, *_ in rows:
        v, t = W.icosphere(int(level))
        assert (len(v), len(t)) == (int(nv), int(nf))
        topo = O.build_topology(t, len(v))
        assert len(topo["edges"]) == 3 * len(t) // 2
        assert len(v) - len(topo["edges"]) + len(t) == 2          # Euler characteristic
        assert bool((topo["wings"][:, 1] >= 0).all())               # closed: every edge has 2 faces


def test_spring_tetra_uniform_expansion_closed_form():
    """Uniform expansion x -> (1+eps) x of a regular tetrahedron stretches
    every edge by eps*l0; summing k(l-l0) e_hat over the three edges of a
    vertex gives F_i = -4 k eps p_i (p_i the rest position)."""
    p, tri = tetra(0.7)
    k, eps = 1.7, 0.013
    b = O.Body(p, tri, np.zeros(3), **only(ks=k))
    x = torch.tensor(p * (1 + eps))
    F = b.internal_forces(x)
    assert torch.allclose(F, torch.tensor(-4.0 * k * eps * p), rtol=1e-12, atol=1e-15)


def test_volume_and_area_tetra_closed_form():
    """Uniform scaling of a regular tetrahedron: by symmetry grad_i V and
    grad_i A are radial and, by homogeneity (degree 3 and 2), sum_i p_i.grad_i V
    = 3V and sum_i p_i.grad_i A = 2A; so F_i = -k_v (V-V0)/V0 * 3V/(4R^2) p_i
    and the global-area force is -k_A (A-A0)/A0 * 2A/(4R^2) p_i."""
    R0, s = 0.9, 1.021
    p, tri = tetra(R0)
    l0 = R0 * math.sqrt(8.0 / 3.0)
    V0, A0 = l0 ** 3 / (6 * math.sqrt(2)), math.sqrt(3) * l0 ** 2
    V, A, R = V0 * s ** 3, A0 * s ** 2, R0 * s
    x = torch.tensor(p * s)
    kv, kA = 2.3, 0.7
    Fv = O.Body(p, tri, np.zeros(3), **only(kv=kv)).internal_forces(x)
    ref = -kv * (V - V0) / V0 * 3 * V / (4 * R * R) * (p * s)
    assert torch.allclose(Fv, torch.tensor(ref), rtol=1e-12, atol=1e-15)
    FA = O.Body(p, tri, np.zeros(3), **only(kA=kA)).internal_forces(x)
    ref = -kA * (A - A0) / A0 * 2 * A / (4 * R * R) * (p * s)
    assert torch.allclose(FA, torch.tensor(ref), rtol=1e-12, atol=1e-15)
    # local area: four equal faces, each with A_f = A/4, A0_f = A0/4
    ka = 1.3
    Fa = O.Body(p, tri, np.zeros(3), **only(ka=ka)).internal_forces(x)
    ref = -ka * (A - A0) / A0 * 2 * A / (4 * R * R) * (p * s)
    assert torch.allclose(Fa, torch.tensor(ref), rtol=1e-12, atol=1e-15)


def hinge_patch(psi, r=0.8):
    """Two triangles on the hinge a=(0,0,0), b=(1,0,0): wing c of face (a,b,c)
    at angle psi about the x axis, wing d of face (b,a,d) fixed at -y."""
    c = np.array([0.4, r * math.cos(psi), r * math.sin(psi)])
    d = np.array([0.55, -1.1, 0.0])
    x = np.array([[0, 0, 0], [1, 0, 0], c, d], dtype=np.float64)
    tri = np.array([[0, 1, 2], [1, 0, 3]], dtype=np.int32)
    return x, tri


def test_bending_hinge_closed_form():
    """Rotating wing c about the hinge by psi changes the dihedral angle by
    exactly -psi (psi>0 lifts c above the plane, folding the outward (+z)
    normals towards each other: a concave fold).  Moving c along x or along
    its radius leaves the angle unchanged.  So F_c = -dW/dc =
    -k_b sin(theta - theta0) dtheta/dpsi * t / r with t the rotation tangent."""
    kb, r = 0.37, 0.8
    rest, tri = hinge_patch(0.0, r)
    b = O.Body(rest, tri, np.zeros(3), closed=False, **only(kb=kb))
    assert float(b.sin0[0]) == pytest.approx(0.0, abs=1e-15)
    for psi in (0.05, -0.3, 0.9):
        x, _ = hinge_patch(psi, r)
        xt = torch.tensor(x)
        cos, sin = O.hinge_angle(xt, b.hinge_edges, b.hinge_wings)
        assert float(sin[0]) == pytest.approx(math.sin(-psi), abs=1e-14)
        assert float(cos[0]) == pytest.approx(math.cos(psi), abs=1e-14)
        F = b.internal_forces(xt)
        theta = -psi
        t = np.array([0.0, -math.sin(psi), math.cos(psi)])
        ref_c = -kb * math.sin(theta) * (-1.0) * t / r
        assert np.allclose(F[2].numpy(), ref_c, rtol=1e-12, atol=1e-15)
        # translation and rotation invariance of W_b
        assert torch.allclose(F.sum(0), torch.zeros(3, dtype=DT), atol=1e-14)
        assert torch.allclose(torch.cross(xt, F, dim=1).sum(0), torch.zeros(3, dtype=DT), atol=1e-14)


def test_bending_convex_ridge_positive():
    """Reading of the sign: on a convex closed surface with outward normals
    every hinge has sin(theta) > 0."""
    v, t = W.icosphere(2)
    b = O.Body(v, t, np.zeros(3))
    assert bool((b.sin0 > 0).all())


def test_bending_rest_angle_zero_flag():
    """theta0 = 0 (literal W_b = k_b(1 - cos theta)): the rest sphere is
    not force free; with the rest angle reading it is."""
    v, t = W.icosphere(2)
    x = torch.tensor(v)
    F0 = O.Body(v, t, np.zeros(3), **only(kb=1.0), theta0_zero=True).internal_forces(x)
    F1 = O.Body(v, t, np.zeros(3), **only(kb=1.0)).internal_forces(x)
    assert float(F0.abs().max()) > 1e-2
    assert float(F1.abs().max()) < 1e-13
    # dihedral angles are scale invariant (homogeneous of degree 0), so the
    # bending virial sum_i x_i . F_i vanishes for any shape
    assert abs(float((F0 * x).sum())) < 1e-12 * float(F0.abs().max()) * len(x)


@pytest.mark.parametrize("kind", ["sphere", "ellipsoid", "sheet"])
def test_zero_force_at_rest(kind):
    """Sec. 5 step 4: at the reference state all internal forces vanish."""
    rng = np.random.default_rng(0)
    if kind == "sheet":
        v, t, bnd = W.elliptic_sheet(0.3, 0.2, 300, rng, jitter=0.2)
        b = O.Body(v, t, np.zeros(3), closed=False, clamped=bnd, ks=2, kb=0.5, ka=1, kA=1, kv=0)
    else:
        v, t = W.icosphere(2)
        if kind == "ellipsoid":
            v = v * np.array([1.0, 1.3, 0.8])
        b = O.Body(0.3 * v, t, np.zeros(3), ks=2, kb=0.5, ka=1, kA=1, kv=1)
    F = b.internal_forces(torch.tensor(b.rest.numpy()))
    assert float(F.abs().max()) < 1e-12


def deformed_body(seed=0, level=2):
    rng = np.random.default_rng(seed)
    v, t = W.icosphere(level)
    rest = 0.2 * v * np.array([1.0, 1.2, 0.9]) + np.array([0.4, 0.5, 0.6])
    b = O.Body(rest, t, np.array([0.4, 0.5, 0.6]), ks=1.3, kb=0.07, ka=0.9, kA=1.1, kv=1.7)
    x = rest * (1 + 0.03 * rng.standard_normal(3)) + 0.01 * rng.standard_normal(rest.shape)
    return b, torch.tensor(x)


def test_momentum_and_angular_momentum_free():
    """All potentials are invariant under translation and rotation, so
    sum F_int = 0 and sum x x F_int = 0 for any deformation."""
    b, x = deformed_body()
    F = b.internal_forces(x)
    scale = float(F.abs().max())
    assert scale > 1e-3
    assert float(F.sum(0).abs().max()) < 1e-13 * scale * len(F)
    assert float(torch.cross(x, F, dim=1).sum(0).abs().max()) < 1e-13 * scale * len(F)


@pytest.mark.parametrize("term", ["We", "Wb", "Wa", "WA", "Wv"])
def test_each_term_vs_central_differences(term):
    """Every force term equals minus the central difference of its energy."""
    b, x = deformed_body(seed=1, level=1)
    xx = x.clone().requires_grad_(True)
    (g,) = torch.autograd.grad(b.energy_terms(xx)[term], xx)
    h = 1e-6
    rng = np.random.default_rng(5)
    for _ in range(6):
        i, d = int(rng.integers(len(x))), int(rng.integers(3))
        xp, xm = x.clone(), x.clone()
        xp[i, d] += h
        xm[i, d] -= h
        fd = (b.energy_terms(xp)[term] - b.energy_terms(xm)[term]) / (2 * h)
        assert float(g[i, d]) == pytest.approx(float(fd), rel=1e-6, abs=1e-9)


def test_volume_homogeneity_and_sphere_limit():
    """V(s x) = s^3 V(x): sum_i x_i . grad_i V = 3 V; and the enclosed
    volume of a fine icosphere approaches 4/3 pi r^3 from below."""
    v, t = W.icosphere(5)
    r = 0.25
    V = float(O.enclosed_volume(torch.tensor(r * v), torch.tensor(t, dtype=torch.long),
                                torch.zeros(3, dtype=DT)))
    exact = 4.0 / 3.0 * math.pi * r ** 3
    assert 0 < exact - V < 2e-3 * exact
    b, x = deformed_body(seed=2)
    xx = (x - b.origin).clone().requires_grad_(True)
    Vx = O.enclosed_volume(xx, b.tri, torch.zeros(3, dtype=DT))
    (g,) = torch.autograd.grad(Vx, xx)
    assert float((g * xx).sum()) == pytest.approx(3.0 * float(Vx), rel=1e-12)


def test_topology_rejects_bad_meshes():
    v, t = W.icosphere(1)
    bad = t.copy()
    bad[0] = bad[0][[0, 2, 1]]          # one face flipped: edge used twice in one direction
    with pytest.raises(O.MeshError):
        O.build_topology(bad, len(v))
    with pytest.raises(O.MeshError):
        O.Body(v, t[:, [0, 2, 1]], np.zeros(3))   # all inward: negative rest volume
