"""Measurement-driven choice of the force-kernel patch size.

A force-kernel block owns a patch of that many vertices and stages the patch
plus its halo in shared memory; small patches repeat more halo work, large
ones hold fewer blocks per SM.  The best size depends on the meshes, so it is
picked by timing the force + node-update kernel (CUDA events between the
launches of ibm_step) on the actual workload.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib

CANDIDATES = (96, 128, 160, 192, 224, 256, 320, 384)


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
