"""The allocation-free body-measures entry point, for callers that cannot
allocate device memory at the point of the call, against the context-based
ibm_body_measures on the same positions, twice in a row (the static scratch
keeps the previous call's contents, so the second call checks that it is
reset).  Collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1612_03399_gb300 import _lib
from paper_1612_03399_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def bodies():
    rng = np.random.default_rng(7)
    b0 = W._sphere_body(2, 0.15, np.array([0.3, 0.4, 0.45]))
    b1 = W._sphere_body(4, 0.12, np.array([0.7, 0.6, 0.4]), rng=rng, stretch=(1.3, 1.0, 0.8))
    sv, st, bnd = W.elliptic_sheet(0.1, 0.07, 700, rng, jitter=0.1)
    c = np.array([0.5, 0.8, 0.6])
    b2 = W.Body(rest=c + sv, tri=st, origin=c, closed=False, clamped=bnd, kv=0.0)
    return [b0, b1, b2]


def test_noalloc_measures_match_context_twice():
    bs = bodies()
    grid = W.Grid((32, 32, 32))
    ctx = _lib.Context(bs, grid)
    lib = _lib.library()
    dev = torch.device("cuda", 0)
    tri = np.concatenate([b.tri + int(ctx.v_off[i]) for i, b in enumerate(bs)]).astype(np.int32)
    tri_d = torch.tensor(tri, device=dev)
    face_off = torch.tensor(np.append(ctx.f_off, ctx.F).astype(np.int32), device=dev)
    closed = torch.tensor([1 if b.closed else 0 for b in bs], dtype=torch.uint8, device=dev)
    max_faces = max(len(b.tri) for b in bs)
    x0, _ = ctx.init_state()
    rng = np.random.default_rng(3)
    for call in range(2):
        x = (x0 * (1.0 + 0.02 * (call + 1))
             + torch.tensor(rng.uniform(-1e-3, 1e-3, tuple(x0.shape)), dtype=torch.float32,
                            device=dev)).contiguous()
        ref = ctx.body_measures(x)
        out = torch.full((len(bs), 2), float("nan"), dtype=torch.float64, device=dev)
        st = lib.ibm_body_measures_noalloc(
            ctypes.c_void_p(x.data_ptr()), ctx.V, ctypes.c_void_p(tri_d.data_ptr()),
            ctypes.c_void_p(face_off.data_ptr()), len(bs), max_faces,
            ctypes.c_void_p(closed.data_ptr()), ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
        assert st == 0, lib.ibm_last_error(None)
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        assert np.allclose(got[:, 0], want[:, 0], rtol=1e-6, atol=0)
        assert np.allclose(got[:, 1], want[:, 1], rtol=1e-6, atol=1e-12)
        assert got[2, 1] == 0.0 and want[2, 1] == 0.0


def test_noalloc_rejects_oversize_requests():
    lib = _lib.library()
    st = lib.ibm_body_measures_noalloc(ctypes.c_void_p(16), 3, ctypes.c_void_p(16),
                                       ctypes.c_void_p(16), 70000, 3, None,
                                       ctypes.c_void_p(16), None)
    assert st == 6
    assert b"static scratch" in lib.ibm_last_error(None)


def _call(lib, x, n_vert, tri_d, face_off, n_bodies, max_faces, closed, out, dev):
    return lib.ibm_body_measures_noalloc(
        ctypes.c_void_p(x.data_ptr()), n_vert, ctypes.c_void_p(tri_d.data_ptr()),
        ctypes.c_void_p(face_off.data_ptr()), n_bodies, max_faces,
        ctypes.c_void_p(closed.data_ptr()) if closed is not None else None,
        ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))


def test_noalloc_flags_bad_caller_data_with_nan():
    """Caller data that would address outside the arrays is caught on the
    device before use: a body with more faces than max_faces_per_body, a body
    with a vertex id outside [0, n_vert) and a body with a reversed face range
    get NaN, the other bodies their exact measures; a body with no faces gets
    (0, 0)."""
    bs = bodies()
    grid = W.Grid((32, 32, 32))
    ctx = _lib.Context(bs, grid)
    lib = _lib.library()
    dev = torch.device("cuda", 0)
    tri = np.concatenate([b.tri + int(ctx.v_off[i]) for i, b in enumerate(bs)]).astype(np.int32)
    fo = np.append(ctx.f_off, ctx.F).astype(np.int32)
    closed = torch.tensor([1 if b.closed else 0 for b in bs], dtype=torch.uint8, device=dev)
    x, _ = ctx.init_state()
    ref = ctx.body_measures(x).cpu().numpy()
    nf = [len(b.tri) for b in bs]
    assert nf[1] > max(nf[0], nf[2])

    # undersized bound: body 1 does not fit, bodies 0 and 2 do
    out = torch.full((3, 2), -1.0, dtype=torch.float64, device=dev)
    st = _call(lib, x, ctx.V, torch.tensor(tri, device=dev), torch.tensor(fo, device=dev), 3,
               max(nf[0], nf[2]), closed, out, dev)
    assert st == 0, lib.ibm_last_error(None)
    got = out.cpu().numpy()
    assert np.isnan(got[1]).all()
    for i in (0, 2):
        assert np.allclose(got[i], ref[i], rtol=1e-6, atol=1e-12)

    # a vertex id one past the end in body 2
    bad = tri.copy()
    bad[fo[2] + 5, 1] = ctx.V
    out.fill_(-1.0)
    st = _call(lib, x, ctx.V, torch.tensor(bad, device=dev), torch.tensor(fo, device=dev), 3,
               max(nf), closed, out, dev)
    assert st == 0
    got = out.cpu().numpy()
    assert np.isnan(got[2]).all()
    for i in (0, 1):
        assert np.allclose(got[i], ref[i], rtol=1e-6, atol=1e-12)

    # an empty body between bodies 0 and 1, and a reversed range after them
    fo5 = np.array([fo[0], fo[1], fo[1], fo[2], fo[1], fo[1]], dtype=np.int32)
    closed5 = torch.tensor([1, 1, 1, 1, 1], dtype=torch.uint8, device=dev)
    out5 = torch.full((5, 2), -1.0, dtype=torch.float64, device=dev)
    st = _call(lib, x, ctx.V, torch.tensor(tri, device=dev), torch.tensor(fo5, device=dev), 5,
               max(nf), closed5, out5, dev)
    assert st == 0
    got = out5.cpu().numpy()
    assert np.allclose(got[0], ref[0], rtol=1e-6, atol=1e-12)
    assert np.array_equal(got[1], [0.0, 0.0])
    assert np.allclose(got[2], ref[1], rtol=1e-6, atol=1e-12)
    assert np.isnan(got[3]).all()
    assert np.array_equal(got[4], [0.0, 0.0])
