"""Measurement-driven choice of the kernels' patch sizes.

A force-kernel block owns a patch of that many vertices and stages the patch
plus its halo in shared memory; small patches repeat more halo work, large
ones hold fewer blocks per SM.  A marker-kernel block owns a surface patch of
128 or 256 faces: the smaller one stages more nodes per face (its row map
has more boundary) but runs twice the blocks with half the shared memory
each.  The best sizes depend on the meshes, so they are picked by timing the
kernels (CUDA events between the launches of ibm_step) on the actual
workload.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib

CANDIDATES = (96, 128, 160, 192, 224, 256, 320, 384)
MARKER_CANDIDATES = (128, 256)


def autotune_patch_size(bodies, grid, fields, dt=1e-3, mu=1.0, alpha=0.3, device=0,
                        candidates=CANDIDATES, steps=6, warmup=2):
    """Return (best patch size, {size: mean force-phase ms})."""
    dev = torch.device("cuda", device)
    n = grid.n
    results = {}
    for P in candidates:
        try:
            ctx = _lib.Context(bodies, grid, dt=dt, mu=mu, alpha=alpha, patch_size=P, device=device,
                               spread_variant=1)
        except _lib.IBMError:
            continue           # patch tables too large for this size
        f = tuple(torch.zeros((n[2], n[1], n[0]), dtype=torch.float32, device=dev) for _ in range(3))
        xa, va = ctx.init_state()
        xb, vb = torch.empty_like(xa), torch.empty_like(va)
        ctx.set_phase_timing(True)
        times = []
        for k in range(warmup + steps):
            ctx.step(xa, va, fields, xb, vb, f)
            if k >= warmup:
                times.append(ctx.phase_times()[3])
            xa, va, xb, vb = xb, vb, xa, va
        ctx.check_device_error()
        results[P] = float(np.mean(times))
        ctx.close()
        del f, xa, va, xb, vb
    best = min(results, key=results.get)
    return best, results


def autotune_marker_patch(bodies, grid, fields, dt=1e-3, mu=1.0, alpha=0.3, device=0,
                          patch_size=0, candidates=MARKER_CANDIDATES, steps=6, warmup=2):
    """Return (best marker patch size, {size: mean ms of footprint clear + marker kernel})."""
    dev = torch.device("cuda", device)
    n = grid.n
    results = {}
    for P in candidates:
        ctx = _lib.Context(bodies, grid, dt=dt, mu=mu, alpha=alpha, patch_size=patch_size,
                           device=device, spread_variant=1, marker_patch=P)
        f = tuple(torch.zeros((n[2], n[1], n[0]), dtype=torch.float32, device=dev) for _ in range(3))
        xa, va = ctx.init_state()
        xb, vb = torch.empty_like(xa), torch.empty_like(va)
        ctx.set_phase_timing(True)
        times = []
        for k in range(warmup + steps):
            ctx.step(xa, va, fields, xb, vb, f)
            if k >= warmup:
                ph = ctx.phase_times()
                times.append(ph[0] + ph[1])
            xa, va, xb, vb = xb, vb, xa, va
        ctx.check_device_error()
        results[P] = float(np.mean(times))
        ctx.close()
        del f, xa, va, xb, vb
    best = min(results, key=results.get)
    # within 1 % (run-to-run noise) the default, 256, is kept
    if 256 in results and results[256] <= 1.01 * results[best]:
        best = 256
    return best, results
