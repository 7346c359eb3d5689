"""Pins of the oracle's per-element constants: van Gelder spring constants for
non-uniform meshes and per-face material maps (reading R18); no GPU.

Van Gelder's edge constants k_e = E t sum_T A_T / l_e^2 make a triangulated
spring sheet respond like a membrane of 2D modulus E t and Poisson ratio 1/3:
under an isotropic stretch (1 + eps) it stores E t eps^2 / (1 - nu) = 1.5 E t
eps^2 per unit area, for ANY triangulation; on an equilateral lattice the
interior constant is sqrt(3)/2 E t (the classical lattice result E = 2k/sqrt3).
"""
import math

import numpy as np
import pytest
import torch

from oracle import ibm_oracle as O
from paper_1612_03399_gb300 import workloads as W

DT = torch.float64


def irregular_sheet(seed=3):
    rng = np.random.default_rng(seed)
    sv, st, bnd = W.elliptic_sheet(0.2, 0.12, 500, rng, jitter=0.3)
    c = np.array([0.5, 0.5, 0.5])
    return c + sv @ W.random_rotation(rng).T, st, c


def ellipsoid(seed=4):
    v, t = W.icosphere(3)
    rng = np.random.default_rng(seed)
    c = np.array([0.5, 0.45, 0.55])
    x = c + (v * np.array([0.3, 0.2, 0.15])) @ W.random_rotation(rng).T
    return x, t, c


def rest_area(x, t):
    return float(0.5 * np.linalg.norm(np.cross(x[t[:, 1]] - x[t[:, 0]], x[t[:, 2]] - x[t[:, 0]]),
                                      axis=1).sum())


@pytest.mark.parametrize("mesh, closed", [(irregular_sheet, False), (ellipsoid, True)])
def test_van_gelder_isotropic_stretch_energy(mesh, closed):
    x, t, c = mesh()
    E = 2.7
    b = O.Body(x, t, c, closed=closed, ks=E, kb=0.0, ka=0.0, kA=0.0, kv=0.0, spring_model=1)
    for eps in (1e-3, 0.05):
        xs = torch.tensor(c + (1.0 + eps) * (x - c), dtype=DT)
        We = float(b.energy_terms(xs)["We"])
        assert We == pytest.approx(1.5 * E * eps ** 2 * rest_area(x, t), rel=1e-12)


def equilateral_patch(rings=5, a=0.01):
    """A hexagonal patch of equilateral triangles of side a."""
    pts, index = [], {}
    for j in range(-rings, rings + 1):
        for i in range(-rings, rings + 1):
            if abs(i) <= rings and abs(j) <= rings and abs(i + j) <= rings:
                index[(i, j)] = len(pts)
                pts.append((a * (i + 0.5 * j), a * (math.sqrt(3) / 2) * j, 0.0))
    tri = []
    for (i, j), k in index.items():
        if (i + 1, j) in index and (i, j + 1) in index:
            tri.append((k, index[(i + 1, j)], index[(i, j + 1)]))
        if (i + 1, j) in index and (i + 1, j - 1) in index:
            tri.append((k, index[(i + 1, j - 1)], index[(i + 1, j)]))
    return np.array(pts) + 0.5, np.array(tri)


def test_van_gelder_equilateral_lattice_constants():
    x, t = equilateral_patch()
    b = O.Body(x, t, np.full(3, 0.5), closed=False, ks=1.0, spring_model=1)
    inner = b.topo["efaces"][:, 1] >= 0
    m = b.m_edge.numpy()
    assert inner.sum() > 0 and (~inner).sum() > 0
    assert np.allclose(m[inner.numpy()], math.sqrt(3) / 2, rtol=1e-12)
    assert np.allclose(m[~inner.numpy()], math.sqrt(3) / 4, rtol=1e-12)


@pytest.mark.parametrize("model", [0, 1])
def test_uniform_material_equals_scaled_constants(model):
    x, t, c = ellipsoid()
    k = dict(ks=1.3, kb=0.07, ka=0.9, kA=0.4, kv=1.1)
    mat = np.tile([2.0, 3.0, 4.0], (len(t), 1))
    b1 = O.Body(x, t, c, spring_model=model, face_material=mat, **k)
    k2 = dict(k, ks=2.0 * k["ks"], kb=3.0 * k["kb"], ka=4.0 * k["ka"])
    b2 = O.Body(x, t, c, spring_model=model, **k2)
    rng = np.random.default_rng(0)
    xs = torch.tensor(x + 0.003 * rng.standard_normal(x.shape), dtype=DT)
    e1, e2 = b1.energy_terms(xs), b2.energy_terms(xs)
    for name in ("We", "Wb", "Wa", "WA", "Wv"):
        assert float(e1[name]) == pytest.approx(float(e2[name]), rel=1e-13)
    assert torch.allclose(b1.internal_forces(xs), b2.internal_forces(xs), rtol=1e-12, atol=1e-15)


def test_two_materials_scale_the_forces_inside_each_region():
    """Springs and bending only; faces with centroid x > x0 have 3x the
    constants.  At a vertex whose faces and whose edges' faces all lie in
    that region the force is exactly 3x the one-material force."""
    x, t, c = irregular_sheet()
    cen = x[t].mean(1)
    x0 = np.median(cen[:, 0])
    mat = np.where((cen[:, 0] > x0)[:, None], 3.0, 1.0) * np.ones((1, 3))
    k = dict(ks=1.0, kb=0.05, ka=0.0, kA=0.0, kv=0.0, closed=False)
    b3 = O.Body(x, t, c, face_material=mat, **k)
    b1 = O.Body(x, t, c, **k)
    rng = np.random.default_rng(1)
    xs = torch.tensor(x + 0.002 * rng.standard_normal(x.shape), dtype=DT)
    F3, F1 = b3.internal_forces(xs).numpy(), b1.internal_forces(xs).numpy()
    # vertices whose 2-ring of faces is entirely in the stiff region
    hi = set(np.where(cen[:, 0] > x0)[0])
    vf = {}
    for f, tri in enumerate(t):
        for v in tri:
            vf.setdefault(int(v), set()).add(f)
    deep = [v for v, fs in vf.items()
            if all(f in hi for f in fs) and all(g in hi for f in fs for w in t[f] for g in vf[int(w)])]
    assert len(deep) > 10
    assert np.allclose(F3[deep], 3.0 * F1[deep], rtol=1e-11, atol=1e-13)
    # and in the soft region the forces are unchanged
    lo = set(range(len(t))) - hi
    soft = [v for v, fs in vf.items()
            if all(f in lo for f in fs) and all(g in lo for f in fs for w in t[f] for g in vf[int(w)])]
    assert len(soft) > 10
    assert np.allclose(F3[soft], F1[soft], rtol=1e-11, atol=1e-13)
