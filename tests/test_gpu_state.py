"""Checkpoint and resume of a context's own state (ibm_get_state /
ibm_set_state) through the C ABI.

The state is what the context keeps between steps: the strong-coupling
history of Hamming's predictor-corrector (Sec. 2.3) and the record of the
grid nodes the last clear-mode step left nonzero in the caller's force
fields.  A second context of the same bodies given the first one's state,
with the caller's arrays as they were, continues the trajectory exactly:
positions and velocities bit for bit, the fields bit for bit with the
tile-owned spread (variant 2) and to float32 rounding with the atomic flush
of variant 1 (its float additions into a node come in any order).  Without
the state the continuation differs (Runge-Kutta steps instead of
predictor-corrector steps; the previous forces are not cleared), so the
tests see the state at work.  Malformed or foreign states are refused before
anything reaches the device."""
import collections
import struct

import numpy as np
import pytest
import torch

from paper_1612_03399_gb300 import _lib

import helpers as H
from test_gpu_parity import mixed_workload

pytestmark = pytest.mark.gpu
DEV = "cuda"
HEADER = struct.Struct("<8sIiqqqq3iIiiiiq")   # the 88-byte header of a state
Header = collections.namedtuple("Header", "magic version variant V F n_chunks n_tiles nx ny nz "
                                          "dt_bits pc_steps pc_have tile_epoch reserved n_rows")


def header(state):
    return Header(*HEADER.unpack_from(state))


def make(wl, variant):
    return _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha,
                        spread_variant=variant)


def zero_fields(wl):
    n = wl.grid.n
    return tuple(torch.zeros((n[2], n[1], n[0]), dtype=torch.float32, device=DEV)
                 for _ in range(3))


def run(ctx, x, v, fields, f, steps, pc):
    for _ in range(steps):
        x1, v1 = torch.empty_like(x), torch.empty_like(v)
        (ctx.step_pc if pc else ctx.step)(x, v, fields, x1, v1, f)
        x, v = x1, v1
    ctx.check_device_error()
    return x, v


def clone(f):
    return tuple(t.clone() for t in f)


def assert_fields(fa, fb, variant):
    for ta, tb in zip(fa, fb):
        if variant == 2:
            assert torch.equal(ta, tb)
        else:
            scale = float(ta.abs().max())
            assert scale > 0
            assert float((ta - tb).abs().max()) <= 1e-6 * scale


@pytest.mark.parametrize("variant", [1, 2])
def test_resume_continues_the_strong_coupling_trajectory(variant):
    wl = mixed_workload()
    fields = H.fields_for(wl, DEV)
    a = make(wl, variant)
    x, v = a.init_state()
    f = zero_fields(wl)
    # five steps: past the three Runge-Kutta start-up steps
    x, v = run(a, x, v, fields, f, 5, True)
    state = a.get_state()
    hdr = header(state)
    assert hdr.magic == b"IBMSTATE" and hdr.pc_steps == 5 and hdr.pc_have == 1
    assert (hdr.nx, hdr.ny, hdr.nz) == tuple(wl.grid.n)
    ck = (x.clone(), v.clone(), clone(f))
    xa, va = run(a, x, v, fields, f, 3, True)

    b = make(wl, variant)
    b.set_state(state)
    fb = clone(ck[2])
    xb, vb = run(b, ck[0], ck[1], fields, fb, 3, True)
    assert torch.equal(xa, xb) and torch.equal(va, vb)
    assert_fields(f, fb, variant)
    # the state read back from the resumed context is the original's, after
    # the same three steps
    assert b.get_state() == a.get_state()

    # without the state the context starts a new trajectory
    c = make(wl, variant)
    xc, vc = run(c, ck[0], ck[1], fields, clone(ck[2]), 3, True)
    assert not torch.equal(xc, xa)


@pytest.mark.parametrize("variant", [1, 2])
def test_resume_clears_the_checkpointed_footprint(variant):
    wl = mixed_workload()
    fields = H.fields_for(wl, DEV)
    a = make(wl, variant)
    x, v = a.init_state()
    f = zero_fields(wl)
    x, v = run(a, x, v, fields, f, 3, False)
    state = a.get_state()
    assert header(state).pc_steps == 0   # no strong-coupling history
    # continue from positions shifted by about seven cells in x, so that the
    # next footprint leaves most of the checkpoint's: those nodes must be
    # zeroed from the footprint record alone
    xs = x.clone()
    xs[0] += 0.2
    ck = (xs, v.clone(), clone(f))
    run(a, xs, v, fields, f, 1, False)

    b = make(wl, variant)
    b.set_state(state)
    fb = clone(ck[2])
    run(b, ck[0], ck[1], fields, fb, 1, False)
    assert_fields(f, fb, variant)

    c = make(wl, variant)
    fc = clone(ck[2])
    run(c, ck[0], ck[1], fields, fc, 1, False)
    stale = max(float((tc - ta).abs().max()) for tc, ta in zip(fc, f))
    assert stale > 1e-3 * max(float(t.abs().max()) for t in ck[2])


def test_state_is_refused_when_malformed_or_foreign():
    wl = mixed_workload()
    fields = H.fields_for(wl, DEV)
    a = make(wl, 1)
    x, v = a.init_state()
    f = zero_fields(wl)
    run(a, x, v, fields, f, 2, False)
    state = a.get_state()
    bad = []
    bad.append(state[:-8])                                   # truncated
    bad.append(b"XBMSTATE" + state[8:])                      # not a state of this library
    # a footprint row that names a row start outside the grid
    hdr = header(state)
    n_chunks, n_rows = hdr.n_chunks, hdr.n_rows
    rows = HEADER.size + 32 * n_chunks
    assert n_rows > 0
    rec = np.frombuffer(state, dtype=np.int32, count=2 * n_rows, offset=rows).reshape(-1, 2)
    k = int(np.nonzero((rec[:, 1] >> 16) > 0)[0][0])
    n = wl.grid.n
    corrupt = bytearray(state)
    struct.pack_into("<i", corrupt, rows + 8 * k, n[0] * n[1] * n[2])
    bad.append(bytes(corrupt))
    b = make(wl, 1)
    for s in bad:
        with pytest.raises(_lib.IBMError, match="ibm_set_state"):
            b.set_state(s)
    # other contexts: another spread variant, another step size, other bodies
    with pytest.raises(_lib.IBMError, match="other bodies"):
        make(wl, 2).set_state(state)
    other = _lib.Context(wl.bodies, wl.grid, dt=wl.dt * 0.5, mu=wl.mu, alpha=wl.alpha,
                         spread_variant=1)
    with pytest.raises(_lib.IBMError, match="other bodies"):
        other.set_state(state)
    wl2 = mixed_workload(n=(40, 40, 32))
    with pytest.raises(_lib.IBMError, match="other bodies"):
        make(wl2, 1).set_state(state)
    # a refused state leaves the context as it was: it still takes a valid one
    b.set_state(state)
    assert b.get_state() == state
