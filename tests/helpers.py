"""Shared test helpers: feed the same seeded inputs to the CUDA library and to
the FP64 oracle, and compare.  Imports both sides; neither side imports this."""
from __future__ import annotations

import math

import numpy as np
import torch

from oracle import ibm_oracle as O
from paper_1612_03399_gb300 import workloads as W

DT = torch.float64


def oracle_bodies(wl, theta0_zero=False):
    return [O.Body(b.rest, b.tri, b.origin, closed=b.closed, clamped=b.clamped, ks=b.ks, kb=b.kb,
                   ka=b.ka, kA=b.kA, kv=b.kv, mass=b.mass, theta0_zero=theta0_zero,
                   spring_model=getattr(b, "spring_model", 0),
                   face_material=getattr(b, "face_material", None))
            for b in wl.bodies]


def oracle_params(wl, forward_euler=False):
    return O.Params(wl.grid.n, wl.grid.L, dt=wl.dt, mu=wl.mu, alpha=wl.alpha,
                    forward_euler=forward_euler)


def split_state(ctx, wl, t):
    """[3, V] float32 device tensor -> per-body [V_b, 3] float64 CPU arrays."""
    a = t.detach().double().cpu().numpy()
    out = []
    for i, b in enumerate(wl.bodies):
        o = int(ctx.v_off[i])
        out.append(a[:, o:o + len(b.rest)].T.copy())
    return out


def split_faces(ctx, wl, t):
    a = t.detach().double().cpu().numpy()
    return [a[:, int(ctx.f_off[i]):int(ctx.f_off[i]) + len(b.tri)].T.copy()
            for i, b in enumerate(wl.bodies)]


def to_abs(wl, rel_list):
    """body-frame positions -> absolute float64 tensors (exact in float64)."""
    return [torch.tensor(r + b.origin) for r, b in zip(rel_list, wl.bodies)]


def state_tensor(wl, arrays, device="cuda"):
    """per-body [V_b, 3] body-frame arrays -> [3, V] float32 device tensor."""
    a = np.concatenate(arrays, 0).T.astype(np.float32)
    return torch.tensor(np.ascontiguousarray(a), device=device)


def rel_positions(wl, abs_list):
    return [x - b.origin for x, b in zip(abs_list, wl.bodies)]


def fields_for(wl, device):
    return W.sample_field(wl.field, wl.grid, device=device, dtype=torch.float32)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def tie_distance(P, grid):
    """Smallest distance, in cells, of points P [M,3] (absolute, float64) from
    a half-cell switch of the nearest-node choice on any of the six lattices
    (offset 0 and 1/2 in each direction)."""
    h = np.array(grid.h)
    t = np.asarray(P) / h
    d = np.full(len(t), np.inf)
    for off in (0.0, 0.5):
        u = t - off
        frac = u - np.floor(u)
        d = np.minimum(d, np.abs(frac - 0.5).min(1))
    return d


def marker_locations(wl, xs_abs, probe_h=None):
    """Centroids and probe ends (both sides) of every face, absolute float64."""
    ph = probe_h if probe_h is not None else sum(wl.grid.h) / 3.0
    pts = []
    for b, x in zip(wl.bodies, xs_abs):
        xx = x.numpy() if torch.is_tensor(x) else x
        tri = b.tri
        xa, xb, xc = xx[tri[:, 0]], xx[tri[:, 1]], xx[tri[:, 2]]
        c = (xa + xb + xc) / 3
        N = np.cross(xb - xa, xc - xa)
        n = N / np.linalg.norm(N, axis=1, keepdims=True)
        pts.append(np.stack([c, c + ph * n, c - ph * n], 1))
    return pts


def tie_free(wl, xs_abs, margin=2e-5):
    """True when no centroid or probe end is within `margin` cells of a
    nearest-node switch (so float32 and float64 pick the same stencils)."""
    for p in marker_locations(wl, xs_abs):
        if tie_distance(p.reshape(-1, 3), wl.grid).min() < margin:
            return False
    return True


def tie_flags(wl, xs_abs, margin=2e-5):
    """Per body: faces whose centroid, and faces whose probe end(s), lie
    within `margin` cells of a nearest-node switch."""
    out = []
    for p in marker_locations(wl, xs_abs):
        d = tie_distance(p.reshape(-1, 3), wl.grid).reshape(-1, 3)
        out.append({"centroid": d[:, 0] < margin, "probe": d[:, 1:].min(1) < margin})
    return out


def tie_mask(wl, xs_abs, margin=2e-5):
    """Per-face boolean (concatenated over bodies): True = safely away from
    every switch."""
    return np.concatenate([tie_distance(p.reshape(-1, 3), wl.grid).reshape(-1, 3).min(1) >= margin
                           for p in marker_locations(wl, xs_abs)])
