"""ctypes binding of the C ABI in include/ibm.h.

Argument marshalling only: every step of the method runs in the CUDA library.
Tensors are passed by data_ptr(); the library never falls back to the CPU and
this module raises if the library or a CUDA device is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

IBM_STEP_CLEAR_PREV = 1

_STATUS = {0: "IBM_OK", 1: "IBM_ERR_INVALID_ARG", 2: "IBM_ERR_MESH", 3: "IBM_ERR_CUDA",
           4: "IBM_ERR_DEVICE", 5: "IBM_ERR_OOM", 6: "IBM_ERR_UNSUPPORTED"}


class IBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class BodyDesc(C.Structure):
    _fields_ = [("n_vert", C.c_int32), ("n_face", C.c_int32),
                ("rest", C.POINTER(C.c_double)), ("tri", C.POINTER(C.c_int32)),
                ("clamped", C.POINTER(C.c_uint8)), ("origin", C.c_double * 3),
                ("ks", C.c_double), ("kb", C.c_double), ("ka", C.c_double), ("kA", C.c_double),
                ("kv", C.c_double), ("mass", C.c_double), ("closed", C.c_int32),
                ("spring_model", C.c_int32), ("face_material", C.POINTER(C.c_float))]


class GridDesc(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("reserved", C.c_int32), ("L", C.c_double * 3)]


class Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("mu", C.c_double), ("alpha", C.c_double),
                ("probe_h", C.c_double), ("theta0_zero", C.c_int32), ("forward_euler", C.c_int32),
                ("patch_size", C.c_int32), ("spread_variant", C.c_int32),
                ("marker_patch", C.c_int32)]


# exported symbols and their signatures (ctypes types), in header order
P = C.c_void_p
SIGNATURES = {
    "ibm_create_bodies": (C.c_int, [C.POINTER(P), C.POINTER(BodyDesc), C.c_int32,
                                    C.POINTER(GridDesc), C.POINTER(Params), C.c_int32]),
    "ibm_destroy": (None, [P]),
    "ibm_last_error": (C.c_char_p, [P]),
    "ibm_set_stream": (C.c_int, [P, P]),
    "ibm_get_sizes": (C.c_int, [P, C.POINTER(C.c_int64)]),
    "ibm_get_params": (C.c_int, [P, C.POINTER(Params)]),
    "ibm_get_offsets": (C.c_int, [P, C.POINTER(C.c_int64)]),
    "ibm_init_state": (C.c_int, [P, P, P]),
    "ibm_set_body_constants": (C.c_int, [P, C.POINTER(C.c_double)]),
    "ibm_body_measures": (C.c_int, [P, P, P]),
    "ibm_compute_forces": (C.c_int, [P, P, P, P]),
    "ibm_interpolate": (C.c_int, [P, P, P, P, P, P, P, P, P, P, P]),
    "ibm_interpolate_fp64": (C.c_int, [P, P, P, P, P, P, P, P, P]),
    "ibm_advance": (C.c_int, [P, P, P, P, P, P, P]),
    "ibm_spread": (C.c_int, [P, P, P, P, P, P]),
    "ibm_step": (C.c_int, [P, P, P, P, P, P, P, P, P, P, P, P, P, C.c_uint32]),
    "ibm_step_pc": (C.c_int, [P, P, P, P, P, P, P, P, P, P, P, P, P, C.c_uint32]),
    "ibm_step_host": (C.c_int, [P, P, P, P, P, P, P, P, P, P, P, P, P, C.c_uint32]),
    "ibm_pc_reset": (C.c_int, [P]),
    "ibm_get_state": (C.c_int, [P, P, C.c_int64, C.POINTER(C.c_int64)]),
    "ibm_set_state": (C.c_int, [P, P, C.c_int64]),
    "ibm_check_device_error": (C.c_int, [P]),
    "ibm_set_phase_timing": (C.c_int, [P, C.c_int32]),
    "ibm_get_phase_times": (C.c_int, [P, C.POINTER(C.c_float)]),
    "ibm_get_counters": (C.c_int, [P, C.POINTER(C.c_int64)]),
    "ibm_backward": (C.c_int, [P, P, P, P, P, P, P, P, P, P, P, P]),
    "ibm_graph_create": (C.c_int, [P, P, P, P, P, P, P, P, P, P, P, P, P, C.c_int32,
                                   C.POINTER(P)]),
    "ibm_graph_launch": (C.c_int, [P]),
    "ibm_graph_destroy": (None, [P]),
    "ibm_taylor_deformation": (C.c_int, [P, P, P]),
    "ibm_taylor_backward": (C.c_int, [P, P, P, P, P]),
    "ibm_body_measures_noalloc": (C.c_int, [P, C.c_int64, P, P, C.c_int32, C.c_int32, P, P, P]),
    "ibm_gts_read": (C.c_int, [C.c_char_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), P, P]),
    "ibm_flow_create": (C.c_int, [C.POINTER(GridDesc), C.c_double, C.c_double, C.POINTER(P)]),
    "ibm_flow_set_stream": (C.c_int, [P, P]),
    "ibm_flow_solve_width": (C.c_int, [P, C.c_int32, C.POINTER(C.c_int32)]),
    "ibm_flow_destroy": (None, [P]),
    "ibm_flow_predict": (C.c_int, [P, C.c_int32, P, P, P, P]),
    "ibm_flow_project": (C.c_int, [P, C.c_int32, P, P, P, P, P, P, P, C.c_float]),
    "ibm_flow_step": (C.c_int, [P, P, P, P, P, P, P, P, P, P, P, P, P]),
    "ibm_flow_set_phase_timing": (C.c_int, [P, C.c_int32]),
    "ibm_flow_get_phase_times": (C.c_int, [P, C.POINTER(C.c_float)]),
}

FLOW_PHASES = ("rhs", "fft_fwd3", "cn_scale", "fft_inv3", "update", "ibm_forcing", "div",
               "fft_fwd1", "poisson_scale", "fft_inv1", "project", "body_marker", "body_force")

_lib = None


def library(build_if_missing: bool = True):
    """Load libibm_gb300.so (building it in-tree first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError(f"{path} not built")
        _build.build()
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(t):
    if t is None:
        return None
    import torch
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _any_ptr(t):
    """Address of a contiguous float32 tensor on the device or the host."""
    import torch
    if not (t.is_contiguous() and t.dtype == torch.float32):
        raise ValueError("expected a contiguous float32 tensor")
    return C.c_void_p(t.data_ptr())


class Context:
    """One set of bodies on one Eulerian grid (ibm_create_bodies).

    bodies: list of workloads.Body; grid: workloads.Grid.  State tensors are
    float32 [3, V] in the body frame (x - origin); per-marker arrays [3, F];
    fields [nz, ny, nx].
    """

    def __init__(self, bodies, grid, dt=1e-3, mu=1.0, alpha=0.3, probe_h=0.0, theta0_zero=False,
                 forward_euler=False, patch_size=0, device=0, spread_variant=0, marker_patch=0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the IBM library needs a CUDA device; there is no CPU fallback")
        self.lib = library()
        self.device = torch.device("cuda", device)
        self._keep = []
        descs = (BodyDesc * len(bodies))()
        for i, b in enumerate(bodies):
            rest = np.ascontiguousarray(b.rest, dtype=np.float64)
            tri = np.ascontiguousarray(b.tri, dtype=np.int32)
            d = descs[i]
            d.n_vert, d.n_face = len(rest), len(tri)
            d.rest = rest.ctypes.data_as(C.POINTER(C.c_double))
            d.tri = tri.ctypes.data_as(C.POINTER(C.c_int32))
            self._keep += [rest, tri]
            if b.clamped is not None:
                cl = np.ascontiguousarray(b.clamped, dtype=np.uint8)
                d.clamped = cl.ctypes.data_as(C.POINTER(C.c_uint8))
                self._keep.append(cl)
            for k in range(3):
                d.origin[k] = float(b.origin[k])
            d.ks, d.kb, d.ka, d.kA, d.kv, d.mass = (float(b.ks), float(b.kb), float(b.ka),
                                                    float(b.kA), float(b.kv), float(b.mass))
            d.closed = 1 if b.closed else 0
            d.spring_model = int(getattr(b, "spring_model", 0))
            fm = getattr(b, "face_material", None)
            if fm is not None:
                fm = np.ascontiguousarray(fm, dtype=np.float32).reshape(len(tri), 3)
                d.face_material = fm.ctypes.data_as(C.POINTER(C.c_float))
                self._keep.append(fm)
        g = GridDesc()
        for k in range(3):
            g.n[k] = int(grid.n[k])
            g.L[k] = float(grid.L[k])
        p = Params(dt=dt, mu=mu, alpha=alpha, probe_h=probe_h, theta0_zero=int(theta0_zero),
                   forward_euler=int(forward_euler), patch_size=int(patch_size),
                   spread_variant=int(spread_variant), marker_patch=int(marker_patch))
        h = C.c_void_p()
        st = self.lib.ibm_create_bodies(C.byref(h), descs, len(bodies), C.byref(g), C.byref(p),
                                        device)
        self._keep = []
        if st != 0:
            raise IBMError(st, self.lib.ibm_last_error(None).decode())
        self.h = h
        sizes = (C.c_int64 * 6)()
        self._check(self.lib.ibm_get_sizes(self.h, sizes))
        self.V, self.F, self.E, self.B, self.n_topo, self.n_work = [int(s) for s in sizes]
        offs = (C.c_int64 * (3 * self.B))()
        self._check(self.lib.ibm_get_offsets(self.h, offs))
        o = np.array(offs, dtype=np.int64).reshape(self.B, 3)
        self.v_off, self.f_off, self.e_off = o[:, 0], o[:, 1], o[:, 2]
        self.grid = grid
        prm = Params()
        self._check(self.lib.ibm_get_params(self.h, C.byref(prm)))
        self.spread_variant = int(prm.spread_variant)
        self.patch_size = int(prm.patch_size)
        self.marker_patch = int(prm.marker_patch)
        self.set_stream(torch.cuda.current_stream(self.device))

    # -- plumbing ------------------------------------------------------------
    def _check(self, st):
        if st != 0:
            raise IBMError(st, self.lib.ibm_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.ibm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self.stream = stream
        self._check(self.lib.ibm_set_stream(self.h, C.c_void_p(stream.cuda_stream)))

    def _vec(self, n):
        import torch
        return torch.empty((3, n), dtype=torch.float32, device=self.device)

    # -- entry points ----------------------------------------------------------
    def init_state(self):
        x, v = self._vec(self.V), self._vec(self.V)
        self._check(self.lib.ibm_init_state(self.h, _ptr(x), _ptr(v)))
        return x, v

    def set_constants(self, consts):
        k = np.ascontiguousarray(consts, dtype=np.float64).reshape(self.B, 6)
        self._check(self.lib.ibm_set_body_constants(self.h, k.ctypes.data_as(C.POINTER(C.c_double))))

    def body_measures(self, x):
        import torch
        out = torch.empty((self.B, 2), dtype=torch.float64, device=self.device)
        self._check(self.lib.ibm_body_measures(self.h, _ptr(x), _ptr(out)))
        return out

    def compute_forces(self, x, energy=False, out=None):
        import torch
        F = out if out is not None else self._vec(self.V)
        E = torch.empty((self.B, 5), dtype=torch.float64, device=self.device) if energy else None
        self._check(self.lib.ibm_compute_forces(self.h, _ptr(x), _ptr(F), _ptr(E)))
        return (F, E) if energy else F

    def interpolate(self, x, v, fields, U=True, F_marker=True, F_ext=True, p=None, accel=None):
        """(U, F_marker, F_ext) per face; p: optional cell-centred pressure
        [nz, ny, nx], accel: optional vertex accelerations [3, V]."""
        u, vv, w = fields
        Uo = self._vec(self.F) if U else None
        Fm = self._vec(self.F) if F_marker else None
        Fe = self._vec(self.F) if F_ext else None
        self._check(self.lib.ibm_interpolate(self.h, _ptr(x), _ptr(v), _ptr(u), _ptr(vv), _ptr(w),
                                             _ptr(p), _ptr(accel), _ptr(Uo), _ptr(Fm), _ptr(Fe)))
        return Uo, Fm, Fe

    def interpolate_fp64(self, x, v, fields, U=True, F_marker=True, F_ext=True):
        """(U, F_marker, F_ext) per face with the float64 general moment solve
        (ibm_interpolate_fp64; no pressure)."""
        u, vv, w = fields
        Uo = self._vec(self.F) if U else None
        Fm = self._vec(self.F) if F_marker else None
        Fe = self._vec(self.F) if F_ext else None
        self._check(self.lib.ibm_interpolate_fp64(self.h, _ptr(x), _ptr(v), _ptr(u), _ptr(vv),
                                                  _ptr(w), _ptr(Uo), _ptr(Fm), _ptr(Fe)))
        return Uo, Fm, Fe

    def advance(self, x, v, F_int, F_ext, x_out=None, v_out=None):
        xo = x_out if x_out is not None else self._vec(self.V)
        vo = v_out if v_out is not None else self._vec(self.V)
        self._check(self.lib.ibm_advance(self.h, _ptr(x), _ptr(v), _ptr(F_int), _ptr(F_ext),
                                         _ptr(xo), _ptr(vo)))
        return xo, vo

    def spread(self, x, F_marker, f):
        fx, fy, fz = f
        self._check(self.lib.ibm_spread(self.h, _ptr(x), _ptr(F_marker), _ptr(fx), _ptr(fy), _ptr(fz)))
        return f

    def step(self, x, v, fields, x_out, v_out, f, clear=True, p=None, accel=None):
        u, vv, w = fields
        fx, fy, fz = f
        self._check(self.lib.ibm_step(self.h, _ptr(x), _ptr(v), _ptr(u), _ptr(vv), _ptr(w),
                                      _ptr(p), _ptr(accel), _ptr(x_out), _ptr(v_out), _ptr(fx),
                                      _ptr(fy), _ptr(fz), IBM_STEP_CLEAR_PREV if clear else 0))

    def step_host(self, x, v, fields, x_out, v_out, f, clear=True, p=None, accel=None):
        """One step with the state (x, v in; x_out, v_out out) in host or
        device tensors (ibm_step_host): the copies between host and device
        are part of the call, which returns when x_out, v_out are written."""
        u, vv, w = fields
        fx, fy, fz = f
        for t in (x, v, x_out, v_out):
            if t.numel() != 3 * self.V:
                raise ValueError("state arrays are [3, V] float32")
        self._check(self.lib.ibm_step_host(self.h, _any_ptr(x), _any_ptr(v), _ptr(u), _ptr(vv),
                                           _ptr(w), _ptr(p), _ptr(accel), _any_ptr(x_out),
                                           _any_ptr(v_out), _ptr(fx), _ptr(fy), _ptr(fz),
                                           IBM_STEP_CLEAR_PREV if clear else 0))

    def step_pc(self, x, v, fields, x_out, v_out, f, clear=True, p=None, accel=None):
        """One Hamming predictor-corrector step (ibm_step_pc); the context
        keeps the history, so (x, v) must be the previous call's outputs."""
        u, vv, w = fields
        fx, fy, fz = f
        self._check(self.lib.ibm_step_pc(self.h, _ptr(x), _ptr(v), _ptr(u), _ptr(vv), _ptr(w),
                                         _ptr(p), _ptr(accel), _ptr(x_out), _ptr(v_out),
                                         _ptr(fx), _ptr(fy), _ptr(fz),
                                         IBM_STEP_CLEAR_PREV if clear else 0))

    def pc_reset(self):
        self._check(self.lib.ibm_pc_reset(self.h))

    def get_state(self):
        """The context's own mutable state (ibm_get_state) as bytes: the
        strong-coupling history and the last clear-mode step's footprint."""
        n = C.c_int64(0)
        self._check(self.lib.ibm_get_state(self.h, None, 0, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(self.lib.ibm_get_state(self.h, C.cast(buf, C.c_void_p), n.value, C.byref(n)))
        return buf.raw[:n.value]

    def set_state(self, state):
        """Restore a state taken by get_state (ibm_set_state)."""
        state = bytes(state)
        self._check(self.lib.ibm_set_state(self.h, state, len(state)))

    def backward(self, x, fields, gx_next, gv_next, p=None, accel=None, v=None, gf=None):
        """Cotangents (gx, gv, gparams [B, 5]) of one step from (x, v)
        (ibm_backward); gf: optional cotangents (gfx, gfy, gfz) of the spread
        force fields, which need v."""
        import torch
        u, vv, w = fields
        gfx, gfy, gfz = gf if gf is not None else (None, None, None)
        gx, gv = self._vec(self.V), self._vec(self.V)
        gp = torch.empty((self.B, 5), dtype=torch.float64, device=self.device)
        self._check(self.lib.ibm_backward(self.h, _ptr(x), _ptr(v), _ptr(u), _ptr(vv), _ptr(w),
                                          _ptr(p), _ptr(accel), _ptr(gx_next), _ptr(gv_next),
                                          _ptr(gfx), _ptr(gfy), _ptr(gfz), _ptr(gx), _ptr(gv),
                                          _ptr(gp)))
        return gx, gv, gp

    def graph(self, xa, va, xb, vb, fields, f, n_steps=2, p=None, accel=None):
        """A StepGraph replaying n_steps ping-pong steps with one launch."""
        return StepGraph(self, xa, va, xb, vb, fields, f, n_steps, p, accel)

    def taylor(self, x):
        """Taylor deformation D [B] (float64) of every closed body at x."""
        import torch
        D = torch.empty(self.B, dtype=torch.float64, device=self.device)
        self._check(self.lib.ibm_taylor_deformation(self.h, _ptr(x), _ptr(D)))
        return D

    def taylor_backward(self, x, gD):
        """gx = d(sum gD D)/dx at x, and D."""
        import torch
        gD = gD.to(device=self.device, dtype=torch.float64).contiguous()
        gx = self._vec(self.V)
        D = torch.empty(self.B, dtype=torch.float64, device=self.device)
        self._check(self.lib.ibm_taylor_backward(self.h, _ptr(x), _ptr(gD), _ptr(gx), _ptr(D)))
        return gx, D

    def check_device_error(self):
        self._check(self.lib.ibm_check_device_error(self.h))

    def set_phase_timing(self, on=True):
        self._check(self.lib.ibm_set_phase_timing(self.h, 1 if on else 0))

    def counters(self):
        out = (C.c_int64 * 4)()
        self._check(self.lib.ibm_get_counters(self.h, out))
        return {"marker_box_fallbacks": int(out[0])}

    def phase_times(self):
        """(clear or set-up, marker, tile-owned spread, force+update)
        milliseconds of the last timed step."""
        ms = (C.c_float * 4)()
        self._check(self.lib.ibm_get_phase_times(self.h, ms))
        return tuple(float(m) for m in ms)


class StepGraph:
    """ibm_graph_create / ibm_graph_launch: n_steps captured steps."""

    def __init__(self, ctx, xa, va, xb, vb, fields, f, n_steps=2, p=None, accel=None):
        self.ctx = ctx
        self._keep = (xa, va, xb, vb, fields, f, p, accel)
        u, vv, w = fields
        fx, fy, fz = f
        h = C.c_void_p()
        ctx._check(ctx.lib.ibm_graph_create(ctx.h, _ptr(xa), _ptr(va), _ptr(xb), _ptr(vb), _ptr(u),
                                            _ptr(vv), _ptr(w), _ptr(p), _ptr(accel), _ptr(fx),
                                            _ptr(fy), _ptr(fz), int(n_steps), C.byref(h)))
        self.h = h
        self.n_steps = n_steps

    def launch(self):
        self.ctx._check(self.ctx.lib.ibm_graph_launch(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.ibm_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Flow:
    """The fluid phase (ibm_flow_*): incompressible Navier-Stokes with the RK3
    fractional step on the periodic MAC grid of `grid` (workloads.Grid).
    Velocity and pressure are caller tensors float32 [nz, ny, nx] updated in
    place; the work arrays and FFT plans belong to the library."""

    def __init__(self, grid, nu, dt, device=0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the flow solver needs a CUDA device; there is no CPU fallback")
        self.lib = library()
        self.device = torch.device("cuda", device)
        g = GridDesc()
        for k in range(3):
            g.n[k] = int(grid.n[k])
            g.L[k] = float(grid.L[k])
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            st = self.lib.ibm_flow_create(C.byref(g), float(nu), float(dt), C.byref(h))
        if st != 0:
            raise IBMError(st, self.lib.ibm_last_error(None).decode())
        self.h = h
        self.grid, self.nu, self.dt = grid, float(nu), float(dt)
        self.set_stream(torch.cuda.current_stream(self.device))

    def _check(self, st, ctx=None):
        if st != 0:
            raise IBMError(st, self.lib.ibm_last_error(None).decode())

    def set_stream(self, stream):
        self.stream = stream
        self._check(self.lib.ibm_flow_set_stream(self.h, C.c_void_p(stream.cuda_stream)))

    def solve_widths(self):
        """Per substep, the half width W of the real-space viscous solve
        (2W + 1 taps per direction), or -1 where it runs in Fourier space."""
        out = []
        for l in range(3):
            w = C.c_int32()
            self._check(self.lib.ibm_flow_solve_width(self.h, l, C.byref(w)))
            out.append(int(w.value))
        return tuple(out)

    def predict(self, substep, fields, p):
        u, vv, w = fields
        self._check(self.lib.ibm_flow_predict(self.h, int(substep), _ptr(u), _ptr(vv), _ptr(w),
                                              _ptr(p)))

    def project(self, substep, fields, p, f=None, f_scale=0.0):
        u, vv, w = fields
        fx, fy, fz = f if f is not None else (None, None, None)
        self._check(self.lib.ibm_flow_project(self.h, int(substep), _ptr(u), _ptr(vv), _ptr(w),
                                              _ptr(p), _ptr(fx), _ptr(fy), _ptr(fz),
                                              float(f_scale)))

    def step(self, fields, p, ctx=None, x=None, v=None, x_out=None, v_out=None, f=None):
        """One coupled step (ibm_flow_step); without ctx the flow alone."""
        u, vv, w = fields
        fx, fy, fz = f if f is not None else (None, None, None)
        self._check(self.lib.ibm_flow_step(self.h, ctx.h if ctx is not None else None, _ptr(x),
                                           _ptr(v), _ptr(x_out), _ptr(v_out), _ptr(u), _ptr(vv),
                                           _ptr(w), _ptr(p), _ptr(fx), _ptr(fy), _ptr(fz)))

    def set_phase_timing(self, on):
        self._check(self.lib.ibm_flow_set_phase_timing(self.h, 1 if on else 0))

    def phase_times(self):
        """Milliseconds per phase of the last timed step (FLOW_PHASES order)."""
        ms = (C.c_float * len(FLOW_PHASES))()
        self._check(self.lib.ibm_flow_get_phase_times(self.h, ms))
        return dict(zip(FLOW_PHASES, (float(m) for m in ms)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.ibm_flow_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
