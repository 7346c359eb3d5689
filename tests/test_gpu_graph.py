"""The CUDA-graph replay of captured steps (ibm_graph_*) reproduces the same
steps launched one by one: positions and velocities bitwise (fixed-order
forces), spread fields bitwise with the tile-owned spread and to float32
summation order with the atomic one."""
import numpy as np
import pytest
import torch

from paper_1612_03399_gb300 import _lib

import helpers as H
from test_gpu_parity import deformed_state, mixed_workload

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.mark.parametrize("variant", [1, 2])
def test_graph_replay_matches_step_by_step(variant):
    wl = mixed_workload()
    fields = H.fields_for(wl, DEV)
    n = wl.grid.n
    zeros = lambda: tuple(torch.zeros((n[2], n[1], n[0]), device=DEV) for _ in range(3))
    x0 = H.state_tensor(wl, deformed_state(wl, 8, scale=0.02, stretch=0.02))
    v0 = torch.zeros_like(x0)
    # step by step
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, spread_variant=variant)
    f1 = zeros()
    xa, va = x0.clone(), v0.clone()
    for _ in range(4):
        xb, vb = torch.empty_like(xa), torch.empty_like(va)
        ctx.step(xa, va, fields, xb, vb, f1)
        xa, va = xb, vb
    # two replays of a 2-step graph
    ctx2 = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, spread_variant=variant)
    f2 = zeros()
    ga, gva = x0.clone(), v0.clone()
    gb, gvb = torch.empty_like(ga), torch.empty_like(gva)
    g = ctx2.graph(ga, gva, gb, gvb, fields, f2, n_steps=2)
    g.launch()
    g.launch()
    torch.cuda.synchronize()
    ctx2.check_device_error()
    assert torch.equal(ga, xa) and torch.equal(gva, va)
    for a, b in zip(f2, f1):
        if variant == 2:
            assert torch.equal(a, b)      # tile-owned spread: bitwise
        else:
            assert torch.allclose(a, b, rtol=1e-5, atol=1e-6 * float(b.abs().max()))
    # a step launched on its own after the replays continues the sequence
    # (the tile-owned spread keeps its bookkeeping on the device)
    xb, vb = torch.empty_like(xa), torch.empty_like(va)
    ctx.step(xa, va, fields, xb, vb, f1)
    hb, hvb = torch.empty_like(ga), torch.empty_like(gva)
    ctx2.step(ga, gva, fields, hb, hvb, f2)
    ctx2.check_device_error()
    assert torch.equal(hb, xb)
    for a, b in zip(f2, f1):
        if variant == 2:
            assert torch.equal(a, b)
        else:
            assert torch.allclose(a, b, rtol=1e-5, atol=1e-6 * float(b.abs().max()))
    g.close()


def test_graph_rejects_odd_step_counts():
    wl = mixed_workload()
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt)
    x, v = ctx.init_state()
    fields = H.fields_for(wl, DEV)
    n = wl.grid.n
    f = tuple(torch.zeros((n[2], n[1], n[0]), device=DEV) for _ in range(3))
    with pytest.raises(_lib.IBMError):
        ctx.graph(x, v, torch.empty_like(x), torch.empty_like(v), fields, f, n_steps=3)
