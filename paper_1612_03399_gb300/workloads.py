"""Seeded synthetic workloads for the Lagrangian IP + MLS-IBM hot path.

This module only *makes inputs*: triangulated bodies (icospheres, stretched
ellipsoids, clamped elliptic leaflet sheets), their placement in the periodic
box, per-body elastic constants, and frozen Eulerian velocity fields sampled
at the staggered (MAC) node positions.  It holds none of the method's
arithmetic (no potentials, no MLS, no spreading, no time stepping), so both the
CUDA path and the FP64 oracle can take their inputs from it.

Workload shapes follow the paper's test cases: spheres discretised into
triangles with the Lagrangian marker at each face centroid (Sec. 2.2,
Fig. lagmesh), 320-face spheres as in the scaling runs (Sec. 5.1), 1280-face
drops (Sec. 3.1), 2562-node drops (Sec. 3.2), and closed/open membranes
(Sec. 4).  Everything is seeded; nothing is read from disk.
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------


def _morton3(p: np.ndarray, bits: int = 10) -> np.ndarray:
    """Morton (Z-order) code of points in [0,1]^3 quantised to 2^bits cells."""
    q = np.clip((p * (1 << bits)).astype(np.int64), 0, (1 << bits) - 1)
    code = np.zeros(len(p), dtype=np.int64)
    for b in range(bits):
        for d in range(3):
            code |= ((q[:, d] >> b) & 1) << (3 * b + d)
    return code


def _reorder_for_locality(verts: np.ndarray, tri: np.ndarray):
    """Relabel vertices and reorder faces along a Z-order curve.

    Nearby vertices get nearby indices, so a contiguous index range is a
    compact surface patch and consecutive faces touch nearby grid cells.
    Orientation of every face is preserved.
    """
    lo, hi = verts.min(0), verts.max(0)
    span = np.maximum(hi - lo, 1e-30)
    vorder = np.argsort(_morton3((verts - lo) / span), kind="stable")
    new_id = np.empty(len(verts), dtype=np.int64)
    new_id[vorder] = np.arange(len(verts))
    verts = verts[vorder]
    tri = new_id[tri]
    cen = verts[tri].mean(1)
    forder = np.argsort(_morton3((cen - lo) / span), kind="stable")
    return verts, tri[forder].astype(np.int32)


def icosphere(level: int):
    """Unit icosphere by `level` midpoint subdivisions of the icosahedron.

    Returns (verts [V,3] float64 on the unit sphere, tri [F,3] int32) with
    V = 10*4^level + 2, F = 20*4^level, faces oriented counter-clockwise seen
    from outside (outward normals).
    """
    v, t = _icosphere_cached(int(level))
    return v.copy(), t.copy()


@functools.lru_cache(maxsize=None)
def _icosphere_cached(level: int):
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    for _ in range(level):
        nv = len(v)
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
        key = np.minimum(e[:, 0], e[:, 1]) * nv + np.maximum(e[:, 0], e[:, 1])
        ukey, inv = np.unique(key, return_inverse=True)
        a, b = ukey // nv, ukey % nv
        mid = v[a] + v[b]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        v = np.concatenate([v, mid])
        nf = len(f)
        m01, m12, m20 = (inv[:nf] + nv, inv[nf:2 * nf] + nv, inv[2 * nf:] + nv)
        f = np.concatenate([
            np.stack([f[:, 0], m01, m20], 1),
            np.stack([f[:, 1], m12, m01], 1),
            np.stack([f[:, 2], m20, m12], 1),
            np.stack([m01, m12, m20], 1)])
    return _reorder_for_locality(v, f)


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniformly random 3x3 rotation matrix (QR of a Gaussian matrix)."""
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def elliptic_sheet(a: float, b: float, target_faces: int, rng: np.random.Generator | None = None,
                   jitter: float = 0.0):
    """Open flat sheet: an equilateral triangular lattice clipped to the
    ellipse (x/a)^2 + (y/b)^2 <= 1 in the z = 0 plane.

    Returns (verts [V,3] float64, tri [F,3] int32, boundary [V] bool).  Faces
    are oriented with normal +z; `boundary` marks vertices on the open edge
    (the clamped nodes of a leaflet).
    """
    area = math.pi * a * b
    h = math.sqrt(4.0 * area / (target_faces * math.sqrt(3.0)))  # equilateral side
    dy = h * math.sqrt(3.0) / 2.0
    ny = int(math.ceil(b / dy)) + 1
    nx = int(math.ceil(a / h)) + 2
    rows = []
    for j in range(-ny, ny + 1):
        off = 0.5 * h * (j & 1)
        xs = (np.arange(-nx, nx + 1) * h + off)
        rows.append(np.stack([xs, np.full_like(xs, j * dy)], 1))
    pts = np.concatenate(rows)
    ncol = 2 * nx + 1
    inside = (pts[:, 0] / a) ** 2 + (pts[:, 1] / b) ** 2 <= 1.0
    tris = []
    for jj in range(2 * ny):
        j = jj - ny
        r0, r1 = jj * ncol, (jj + 1) * ncol
        for i in range(ncol - 1):
            if (j & 1) == 0:   # row j even: upper row shifted right
                t1 = (r0 + i, r0 + i + 1, r1 + i)
                t2 = (r0 + i + 1, r1 + i + 1, r1 + i)
            else:
                t1 = (r0 + i, r0 + i + 1, r1 + i + 1)
                t2 = (r0 + i, r1 + i + 1, r1 + i)
            tris.append(t1)
            tris.append(t2)
    tris = np.array(tris, dtype=np.int64)
    keep = inside[tris].all(1)
    tris = tris[keep]
    used = np.unique(tris)
    remap = -np.ones(len(pts), dtype=np.int64)
    remap[used] = np.arange(len(used))
    tris = remap[tris]
    v2 = pts[used]
    verts = np.concatenate([v2, np.zeros((len(v2), 1))], 1)
    # orientation: make every normal +z
    e1 = verts[tris[:, 1]] - verts[tris[:, 0]]
    e2 = verts[tris[:, 2]] - verts[tris[:, 0]]
    nz = e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0]
    flip = nz < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    # boundary vertices: endpoints of edges used by exactly one face
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
    key = np.minimum(e[:, 0], e[:, 1]) * len(verts) + np.maximum(e[:, 0], e[:, 1])
    uk, cnt = np.unique(key, return_counts=True)
    bkey = uk[cnt == 1]
    boundary = np.zeros(len(verts), dtype=bool)
    boundary[bkey // len(verts)] = True
    boundary[bkey % len(verts)] = True
    if jitter > 0.0 and rng is not None:
        interior = ~boundary
        verts[interior, :2] += jitter * h * rng.uniform(-1, 1, (interior.sum(), 2))
    verts, tris = _reorder_for_locality_keep(verts, tris, boundary)
    return verts[0], tris, verts[1]


def _reorder_for_locality_keep(verts, tris, flags):
    lo, hi = verts.min(0), verts.max(0)
    span = np.maximum(hi - lo, 1e-30)
    vorder = np.argsort(_morton3((verts - lo) / span), kind="stable")
    new_id = np.empty(len(verts), dtype=np.int64)
    new_id[vorder] = np.arange(len(verts))
    v = verts[vorder]
    fl = flags[vorder]
    t = new_id[tris]
    cen = v[t].mean(1)
    forder = np.argsort(_morton3((cen - lo) / span), kind="stable")
    return (v, fl), t[forder].astype(np.int32)


# --------------------------------------------------------------------------
# bodies, grid, workload containers
# --------------------------------------------------------------------------


@dataclass
class Body:
    """One triangulated body.  `rest` is the absolute rest (and initial)
    position of every vertex, `origin` the body-frame origin used to store
    positions relative to the body (a point near the body centre)."""
    rest: np.ndarray                 # [V,3] float64, absolute
    tri: np.ndarray                  # [F,3] int32, outward CCW
    origin: np.ndarray               # [3] float64
    closed: bool = True
    clamped: np.ndarray | None = None  # [V] bool
    ks: float = 1.0
    kb: float = 0.01
    ka: float = 1.0                  # local (per face) area constant
    kA: float = 1.0                  # global (per body) area constant
    kv: float = 1.0                  # volume constant (closed bodies)
    mass: float = 1.0
    level: int = -1                  # icosphere level, -1 for other meshes
    radius: float = 0.0              # bounding radius about `origin`
    spring_model: int = 0            # 0 uniform k_e = ks, 1 van Gelder (ks = E t)
    face_material: np.ndarray | None = None  # [F,3] multipliers of (ks, kb, ka)


@dataclass
class Grid:
    """Triply periodic box [0,L)^3 with n^3 cells, MAC-staggered velocity."""
    n: tuple
    L: tuple = (1.0, 1.0, 1.0)

    @property
    def h(self):
        return tuple(self.L[d] / self.n[d] for d in range(3))


@dataclass
class Workload:
    name: str
    bodies: list
    grid: Grid
    field: dict                      # {"kind": "shear"} or {"kind": "fourier", modes...}
    dt: float = 1e-3
    steps: int = 100
    mu: float = 1.0
    alpha: float = 0.3
    seed: int = 0
    notes: dict = field(default_factory=dict)

    @property
    def n_vert(self):
        return sum(len(b.rest) for b in self.bodies)

    @property
    def n_face(self):
        return sum(len(b.tri) for b in self.bodies)


# --------------------------------------------------------------------------
# placement
# --------------------------------------------------------------------------


def poisson_disk(radii: np.ndarray, gap: float, rng: np.random.Generator, box: float = 1.0,
                 y_margin: bool = False, max_tries: int = 200):
    """Seeded dart throwing of non-overlapping spheres in the periodic box.

    Sphere i (bounding radius radii[i]) keeps distance >= r_i + r_j + gap to
    every other (minimum-image distance).  Largest first.  If `y_margin`, the
    sphere plus `gap` must not cross the y = 0 / y = box seam (for a linear
    shear field, which is discontinuous there).  If no spot is found after
    `max_tries` darts the gap is halved for that sphere (recorded in the
    returned `relaxed` count); overlap never affects correctness or cost.
    """
    n = len(radii)
    order = np.argsort(-radii, kind="stable")
    centres = np.zeros((n, 3))
    cell = max(2.0 * radii.max() + gap, 1e-3)
    ncell = max(1, int(box / cell))
    cell = box / ncell
    buckets: dict = {}
    relaxed = 0
    rmax = radii.max()
    for i in order:
        r = radii[i]
        g = gap
        placed = False
        while not placed:
            for _ in range(max_tries):
                c = rng.uniform(0.0, box, 3)
                if y_margin:
                    lo = r + gap
                    c[1] = rng.uniform(lo, box - lo)
                ci = (c / cell).astype(int) % ncell
                reach = int(math.ceil((r + rmax + g) / cell))
                reach = min(reach, ncell // 2)
                ok = True
                for dx in range(-reach, reach + 1):
                    for dy in range(-reach, reach + 1):
                        for dz in range(-reach, reach + 1):
                            key = ((ci[0] + dx) % ncell, (ci[1] + dy) % ncell, (ci[2] + dz) % ncell)
                            for j in buckets.get(key, ()):
                                d = c - centres[j]
                                d -= box * np.round(d / box)
                                if d @ d < (r + radii[j] + g) ** 2:
                                    ok = False
                                    break
                            if not ok:
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if ok:
                    centres[i] = c
                    buckets.setdefault(tuple(ci), []).append(i)
                    placed = True
                    break
            if not placed:
                g *= 0.5
                relaxed += 1
                if g < 1e-9:
                    g = -1e9   # give up on spacing entirely
    return centres, relaxed


# --------------------------------------------------------------------------
# frozen Eulerian velocity
# --------------------------------------------------------------------------


def fourier_modes(n_modes: int, kmax: int, amplitude: float, rng: np.random.Generator):
    """Random divergence-free Fourier modes u(x) = sum_m a_m sin(2 pi k_m.x + p_m)
    with integer wavevectors 1 <= |k_m| <= kmax, a_m perpendicular to k_m and
    |a_m| = amplitude, phases uniform in [0, 2 pi)."""
    ks, amps = [], []
    while len(ks) < n_modes:
        k = rng.integers(-kmax, kmax + 1, 3)
        nk = np.linalg.norm(k)
        if nk < 1.0 or nk > kmax:
            continue
        a = rng.standard_normal(3)
        kh = k / nk
        a -= (a @ kh) * kh
        a *= amplitude / np.linalg.norm(a)
        ks.append(k)
        amps.append(a)
    phase = rng.uniform(0.0, 2.0 * math.pi, n_modes)
    return {"kind": "fourier", "k": np.array(ks, dtype=np.int64), "a": np.array(amps),
            "phase": phase}


MAC_OFFSET = ((0.0, 0.5, 0.5), (0.5, 0.0, 0.5), (0.5, 0.5, 0.0))
"""Node offsets, in cells, of the u, v, w lattices of the staggered grid: u at
(i, j+1/2, k+1/2) h, v at (i+1/2, j, k+1/2) h, w at (i+1/2, j+1/2, k) h."""


def sample_field(spec: dict, grid: Grid, device="cpu", dtype=None):
    """Velocity components (u, v, w), each a [nz, ny, nx] tensor (x fastest),
    evaluated at that component's MAC node positions.

    `spec` is {"kind": "shear"} (u = y - L_y/2, v = w = 0), {"kind":
    "uniform", "U": (U0, U1, U2)} or a fourier_modes() dict.
    """
    import torch
    dtype = dtype or torch.float32
    nx, ny, nz = grid.n
    hx, hy, hz = grid.h
    out = []
    for comp in range(3):
        off = MAC_OFFSET[comp]
        x = (torch.arange(nx, dtype=torch.float64, device=device) + off[0]) * hx
        y = (torch.arange(ny, dtype=torch.float64, device=device) + off[1]) * hy
        z = (torch.arange(nz, dtype=torch.float64, device=device) + off[2]) * hz
        if spec["kind"] == "shear":
            if comp == 0:
                f = (y - 0.5 * grid.L[1]).view(1, ny, 1).expand(nz, ny, nx)
            else:
                f = torch.zeros((nz, ny, nx), dtype=torch.float64, device=device)
            out.append(f.to(dtype).contiguous())
            continue
        if spec["kind"] == "uniform":
            out.append(torch.full((nz, ny, nx), float(spec["U"][comp]), dtype=dtype, device=device))
            continue
        if spec["kind"] == "linear":
            g = np.asarray(spec["G"], dtype=np.float64)   # u_i = c_i + sum_j G_ij x_j
            c = np.asarray(spec["c"], dtype=np.float64)
            f = (c[comp] + g[comp, 0] * x.view(1, 1, nx) + g[comp, 1] * y.view(1, ny, 1)
                 + g[comp, 2] * z.view(nz, 1, 1)).expand(nz, ny, nx)
            out.append(f.to(dtype).contiguous())
            continue
        # sum of separable complex exponentials, imaginary part
        cdt = torch.complex128 if dtype == torch.float64 else torch.complex64
        acc = torch.zeros((nz, ny, nx), dtype=dtype, device=device)
        for m in range(len(spec["phase"])):
            k = spec["k"][m]
            a = float(spec["a"][m][comp])
            if a == 0.0:
                continue
            ex = torch.exp(1j * (2 * math.pi * k[0] / grid.L[0]) * x).to(cdt)
            ey = torch.exp(1j * (2 * math.pi * k[1] / grid.L[1]) * y).to(cdt)
            ez = torch.exp(1j * ((2 * math.pi * k[2] / grid.L[2]) * z + float(spec["phase"][m]))).to(cdt)
            plane = (ez.view(nz, 1) * ey.view(1, ny)) * a
            acc += (plane.view(nz, ny, 1) * ex.view(1, 1, nx)).imag.to(dtype)
        out.append(acc.contiguous())
    return tuple(out)


PRESSURE_OFFSET = (0.5, 0.5, 0.5)
"""Node offsets, in cells, of the pressure lattice: cell centres."""


def pressure_modes(n_modes: int, kmax: int, amplitude: float, rng: np.random.Generator):
    """Random scalar Fourier modes p(x) = sum_m a_m sin(2 pi k_m.x + p_m),
    integer wavevectors 1 <= |k_m| <= kmax, amplitudes a_m = amplitude * U[-1, 1]."""
    ks = []
    while len(ks) < n_modes:
        k = rng.integers(-kmax, kmax + 1, 3)
        if 1.0 <= np.linalg.norm(k) <= kmax:
            ks.append(k)
    a = amplitude * rng.uniform(-1.0, 1.0, n_modes)
    phase = rng.uniform(0.0, 2.0 * math.pi, n_modes)
    return {"kind": "fourier", "k": np.array(ks, dtype=np.int64), "a": a, "phase": phase}


def sample_pressure(spec: dict, grid: Grid, device="cpu", dtype=None):
    """A scalar field [nz, ny, nx] at the cell centres: {"kind": "uniform",
    "p": p0}, {"kind": "linear", "p": p0, "G": (gx, gy, gz)} (p = p0 + G.x) or
    a pressure_modes() dict."""
    import torch
    dtype = dtype or torch.float32
    nx, ny, nz = grid.n
    hx, hy, hz = grid.h
    off = PRESSURE_OFFSET
    x = (torch.arange(nx, dtype=torch.float64, device=device) + off[0]) * hx
    y = (torch.arange(ny, dtype=torch.float64, device=device) + off[1]) * hy
    z = (torch.arange(nz, dtype=torch.float64, device=device) + off[2]) * hz
    if spec["kind"] == "uniform":
        return torch.full((nz, ny, nx), float(spec["p"]), dtype=dtype, device=device)
    if spec["kind"] == "linear":
        g = [float(v) for v in spec["G"]]
        f = (float(spec["p"]) + g[0] * x.view(1, 1, nx) + g[1] * y.view(1, ny, 1)
             + g[2] * z.view(nz, 1, 1)).expand(nz, ny, nx)
        return f.to(dtype).contiguous()
    cdt = torch.complex128 if dtype == torch.float64 else torch.complex64
    acc = torch.zeros((nz, ny, nx), dtype=dtype, device=device)
    for m in range(len(spec["phase"])):
        k = spec["k"][m]
        a = float(spec["a"][m])
        ex = torch.exp(1j * (2 * math.pi * k[0] / grid.L[0]) * x).to(cdt)
        ey = torch.exp(1j * (2 * math.pi * k[1] / grid.L[1]) * y).to(cdt)
        ez = torch.exp(1j * ((2 * math.pi * k[2] / grid.L[2]) * z + float(spec["phase"][m]))).to(cdt)
        plane = (ez.view(nz, 1) * ey.view(1, ny)) * a
        acc += (plane.view(nz, ny, 1) * ex.view(1, 1, nx)).imag.to(dtype)
    return acc.contiguous()


# --------------------------------------------------------------------------
# named workloads (the benchmarked configurations and their small variants)
# --------------------------------------------------------------------------


def _sphere_body(level, radius, centre, rng=None, stretch=None, **params):
    v, t = icosphere(level)
    if stretch is not None:
        rot = random_rotation(rng)
        ax = np.asarray(stretch)
        v = ((v @ rot) * ax) @ rot.T
    rest = centre + radius * v
    b = Body(rest=rest, tri=t, origin=np.array(centre, dtype=np.float64), level=level,
             radius=radius * (max(stretch) if stretch is not None else 1.0), **params)
    return b


def single_drop(level=3, n=64, radius=0.25, seed=0, steps=100):
    """One spherical drop (icosphere) in the middle of the unit box under the
    frozen linear shear u = y - 0.5 (the paper's drop-in-shear set-up,
    Sec. 3.1, with the flow frozen)."""
    body = _sphere_body(level, radius, np.array([0.5, 0.5, 0.5]), ks=1.0, kb=0.01,
                        ka=1.0, kA=1.0, kv=1.0, mass=1.0)
    return Workload(name=f"drop_L{level}_n{n}", bodies=[body], grid=Grid((n, n, n)),
                    field={"kind": "shear"}, steps=steps, seed=seed)


def batched_drops(n_bodies=1000, level=3, n=512, rmin=0.015, rmax=0.03, seed=1, steps=200,
                  n_modes=32, kmax=8, amplitude=1.0):
    """Many equal-topology drops: radii uniform in [rmin, rmax], centres by
    Poisson-disk dart throwing (gap 3 cells), k_s ~ U[0.5, 2],
    k_b ~ U[0.005, 0.02] per body, random divergence-free Fourier velocity."""
    rng = np.random.default_rng(seed)
    radii = rng.uniform(rmin, rmax, n_bodies)
    centres, relaxed = poisson_disk(radii, 3.0 / n, rng)
    ks = rng.uniform(0.5, 2.0, n_bodies)
    kb = rng.uniform(0.005, 0.02, n_bodies)
    bodies = [_sphere_body(level, radii[i], centres[i], ks=ks[i], kb=kb[i], ka=1.0, kA=1.0,
                           kv=1.0, mass=1.0) for i in range(n_bodies)]
    fld = fourier_modes(n_modes, kmax, amplitude, rng)
    return Workload(name=f"drops{n_bodies}_L{level}_n{n}", bodies=bodies, grid=Grid((n, n, n)),
                    field=fld, steps=steps, seed=seed, notes={"relaxed_placements": relaxed})


def uneven_bodies(n_bodies=4096, n=768, seed=2, steps=200, levels=(2, 3, 4, 5),
                  probs=(0.4, 0.3, 0.2, 0.1), rbase=0.005, n_modes=32, kmax=8, amplitude=1.0):
    """Closed bodies of uneven size: icosphere levels drawn with the given
    probabilities, radius rbase * 2^(level - levels[0]), rest shapes stretched
    into ellipsoids with axis ratios U[1, 1.5] along a random orientation."""
    rng = np.random.default_rng(seed)
    lev = rng.choice(np.array(levels), size=n_bodies, p=np.array(probs))
    radii = rbase * 2.0 ** (lev - levels[0])
    stretch = rng.uniform(1.0, 1.5, (n_bodies, 3))
    bound = radii * stretch.max(1)
    centres, relaxed = poisson_disk(bound, 3.0 / n, rng)
    ks = rng.uniform(0.5, 2.0, n_bodies)
    kb = rng.uniform(0.005, 0.02, n_bodies)
    bodies = [_sphere_body(int(lev[i]), radii[i], centres[i], rng=rng, stretch=stretch[i],
                           ks=ks[i], kb=kb[i], ka=1.0, kA=1.0, kv=1.0, mass=1.0)
              for i in range(n_bodies)]
    fld = fourier_modes(n_modes, kmax, amplitude, rng)
    return Workload(name=f"uneven{n_bodies}_n{n}", bodies=bodies, grid=Grid((n, n, n)),
                    field=fld, steps=steps, seed=seed, notes={"relaxed_placements": relaxed})


def shear_drops(n_bodies=256, level=4, n=256, radius=0.04, seed=3, steps=50):
    """Equal drops in frozen linear shear, kept clear of the y seam, with a
    seeded target Taylor deformation D* ~ U[0.05, 0.3] per drop."""
    rng = np.random.default_rng(seed)
    radii = np.full(n_bodies, radius)
    centres, relaxed = poisson_disk(radii, 3.0 / n + 2.5 / n, rng, y_margin=True)
    bodies = [_sphere_body(level, radius, centres[i], ks=1.0, kb=0.01, ka=1.0, kA=1.0, kv=1.0,
                           mass=1.0) for i in range(n_bodies)]
    target = rng.uniform(0.05, 0.3, n_bodies)
    return Workload(name=f"shear{n_bodies}_L{level}_n{n}", bodies=bodies, grid=Grid((n, n, n)),
                    field={"kind": "shear"}, steps=steps, seed=seed,
                    notes={"D_target": target, "relaxed_placements": relaxed})


def membranes(level=8, n=512, leaflet_faces=100_000, seed=4, steps=100, dt=1e-4):
    """One closed ellipsoidal membrane (semi-axes 0.3, 0.3, 0.45) plus two
    clamped elliptic leaflet sheets (semi-axes 0.12, 0.08) at z = 0.5 +- 0.1
    inside it; Fourier velocity with amplitude 2.

    dt = 1e-4: the leaflets' edges (about 8e-4) make their stiffest bending
    mode omega ~ 7e3 for unit node mass, and the explicit step needs
    omega dt < 2 (dt = 1e-3 would give 7.3)."""
    rng = np.random.default_rng(seed)
    v, t = icosphere(level)
    c = np.array([0.5, 0.5, 0.5])
    memb = Body(rest=c + v * np.array([0.3, 0.3, 0.45]), tri=t, origin=c.copy(), closed=True,
                ks=10.0, kb=0.1, ka=1.0, kA=1.0, kv=1.0, level=level, radius=0.45)
    bodies = [memb]
    for dz in (-0.1, 0.1):
        sv, st, bnd = elliptic_sheet(0.12, 0.08, leaflet_faces, rng, jitter=0.1)
        oc = c + np.array([0.0, 0.0, dz])
        bodies.append(Body(rest=oc + sv, tri=st, origin=oc, closed=False, clamped=bnd,
                           ks=10.0, kb=1.0, ka=1.0, kA=0.0, kv=0.0, radius=0.12))
    fld = fourier_modes(32, 8, 2.0, rng)
    return Workload(name=f"membranes_L{level}_n{n}", bodies=bodies, grid=Grid((n, n, n)),
                    field=fld, steps=steps, seed=seed, dt=dt)


def perturb_positions(wl: Workload, scale: float, seed: int, stretch: float = 0.0):
    """Deformed copies of every body's rest positions (absolute, float64):
    a global stretch (1 + stretch) along a random axis about the body origin
    plus uniform random displacements of `scale` times the body's mean edge
    length.  Clamped nodes are left at rest.  Used to exercise the internal
    forces away from the rest state."""
    rng = np.random.default_rng(seed)
    out = []
    for b in wl.bodies:
        x = b.rest.copy()
        if stretch:
            ax = rng.standard_normal(3)
            ax /= np.linalg.norm(ax)
            rel = x - b.origin
            x = b.origin + rel + stretch * np.outer(rel @ ax, ax)
        e = b.rest[b.tri[:, 1]] - b.rest[b.tri[:, 0]]
        lmean = np.linalg.norm(e, axis=1).mean()
        d = scale * lmean * rng.uniform(-1, 1, x.shape)
        if b.clamped is not None:
            d[b.clamped] = 0.0
            if stretch:
                x[b.clamped] = b.rest[b.clamped]
        out.append(x + d)
    return out
