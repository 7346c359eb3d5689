"""ibm_step_host through the C ABI: the step with the body state in host
memory (page-locked or ordinary) or on the device, in any mix, gives the
same results as ibm_step on device arrays: positions and velocities bit for
bit over several steps, the spread fields bit for bit with the tile-owned
spread (variant 2) and to float32 summation order with variant 1."""
import pytest
import torch

from paper_1612_03399_gb300 import _lib
from paper_1612_03399_gb300 import workloads as W

import helpers as H
from test_gpu_parity import mixed_workload

pytestmark = pytest.mark.gpu
DEV = "cuda"
STEPS = 3


def zero_fields(wl):
    n = wl.grid.n
    return tuple(torch.zeros((n[2], n[1], n[0]), dtype=torch.float32, device=DEV)
                 for _ in range(3))


def place(t, where):
    if where == "device":
        return t.to(DEV).clone()
    h = t.cpu().clone()
    return h.pin_memory() if where == "pinned" else h


def assert_fields(fa, fb, variant):
    for ta, tb in zip(fa, fb):
        if variant == 2:
            assert torch.equal(ta, tb)
        else:
            assert float((ta - tb).abs().max()) <= 1e-6 * float(ta.abs().max())


@pytest.mark.parametrize("variant,where_in,where_out",
                         [(1, "pinned", "pinned"), (2, "pinned", "pinned"),
                          (1, "pageable", "pageable"), (1, "device", "pinned"),
                          (2, "pinned", "device")])
def test_host_step_matches_device_step(variant, where_in, where_out):
    wl = mixed_workload()
    fields = H.fields_for(wl, DEV)
    a = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha,
                     spread_variant=variant)
    b = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha,
                     spread_variant=variant)
    x, v = a.init_state()
    fa, fb = zero_fields(wl), zero_fields(wl)
    xh, vh = place(x, where_in), place(v, where_in)
    for _ in range(STEPS):
        x1, v1 = torch.empty_like(x), torch.empty_like(v)
        a.step(x, v, fields, x1, v1, fa)
        xo, vo = place(torch.empty_like(x), where_out), place(torch.empty_like(v), where_out)
        b.step_host(xh, vh, fields, xo, vo, fb)
        # the call is synchronous: the outputs are complete on return
        assert torch.equal(xo.to(DEV), x1) and torch.equal(vo.to(DEV), v1)
        x, v = x1, v1
        xh, vh = (xo, vo) if where_in == where_out else (place(xo, where_in), place(vo, where_in))
    a.check_device_error()
    b.check_device_error()
    assert_fields(fa, fb, variant)


@pytest.mark.parametrize("patch", [96, 224])
def test_host_step_many_mirror_chunks(patch):
    """40 drops: the outputs span 38 chunks of the host mirror, and the runs
    of own vertices of the force patches straddle chunk boundaries."""
    wl = W.batched_drops(40, 3, 128, seed=3)
    fields = W.sample_field(wl.field, wl.grid, device=DEV, dtype=torch.float32)
    a = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha, patch_size=patch)
    b = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha, patch_size=patch)
    x, v = a.init_state()
    fa, fb = zero_fields(wl), zero_fields(wl)
    xh, vh = x.cpu().pin_memory(), v.cpu().pin_memory()
    for _ in range(STEPS):
        x1, v1 = torch.empty_like(x), torch.empty_like(v)
        a.step(x, v, fields, x1, v1, fa)
        xo, vo = torch.empty_like(xh).pin_memory(), torch.empty_like(vh).pin_memory()
        b.step_host(xh, vh, fields, xo, vo, fb)
        assert torch.equal(xo.to(DEV), x1) and torch.equal(vo.to(DEV), v1)
        x, v, xh, vh = x1, v1, xo, vo
    b.check_device_error()
    assert_fields(fa, fb, 1)


def test_host_step_refuses_aliased_outputs():
    wl = mixed_workload()
    fields = H.fields_for(wl, DEV)
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    x, v = ctx.init_state()
    xh, vh = x.cpu().pin_memory(), v.cpu().pin_memory()
    with pytest.raises(_lib.IBMError, match="alias"):
        ctx.step_host(xh, vh, fields, xh, torch.empty_like(vh), zero_fields(wl))
