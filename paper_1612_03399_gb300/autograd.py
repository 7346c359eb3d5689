"""torch.autograd integration of the library's hand-written adjoints.

`rollout` runs n steps of the Lagrangian step (ibm_step) and is
differentiable with respect to the initial positions and velocities and the
per-body elastic constants (k_s, k_b, k_a, k_A, k_v); its backward pass uses
segment checkpointing: the forward keeps only the state at the start of every
segment, and the backward recomputes each segment's states before stepping
back through them with ibm_backward.  `taylor_deformation` is the drop
deformation D = (L - B)/(L + B) of Sec. 3.1 with its adjoint
(ibm_taylor_backward).  Together they let the paper's ad-hoc elastic
constants be fitted by gradient descent to a target deformation.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib
from . import workloads as W

CONSTANTS = ("ks", "kb", "ka", "kA", "kv")


class Simulation:
    """A context, its frozen velocity field and a scratch force field."""

    def __init__(self, bodies, grid, field_spec, dt=1e-3, mu=1.0, alpha=0.3, device=0, **kw):
        self.ctx = _lib.Context(bodies, grid, dt=dt, mu=mu, alpha=alpha, device=device, **kw)
        dev = self.ctx.device
        self.fields = W.sample_field(field_spec, grid, device=dev, dtype=torch.float32)
        nx, ny, nz = grid.n
        self.f = tuple(torch.zeros((nz, ny, nx), dtype=torch.float32, device=dev) for _ in range(3))
        self.base = np.array([[b.ks, b.kb, b.ka, b.kA, b.kv, b.mass] for b in bodies],
                             dtype=np.float64)
        self._k = None

    def constants(self):
        """The current (k_s, k_b, k_a, k_A, k_v) per body as a [B, 5] float64 tensor."""
        return torch.tensor(self.base[:, :5], dtype=torch.float64)

    def set_constants(self, k):
        kk = k.detach().to("cpu", torch.float64).numpy()
        if self._k is not None and np.array_equal(kk, self._k):
            return
        full = self.base.copy()
        full[:, :5] = kk
        self.ctx.set_constants(full)
        self._k = kk.copy()

    def step(self, x, v):
        x1, v1 = torch.empty_like(x), torch.empty_like(v)
        self.ctx.step(x, v, self.fields, x1, v1, self.f)
        return x1, v1


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(fctx, x0, v0, k, sim, n_steps, every):
        sim.set_constants(k)
        x, v = x0.detach().contiguous(), v0.detach().contiguous()
        starts = []
        for s in range(n_steps):
            if s % every == 0:
                starts.append((x, v))
            x, v = sim.step(x, v)
        fctx.sim, fctx.starts, fctx.n, fctx.every = sim, starts, n_steps, every
        fctx.save_for_backward(k)
        return x, v

    @staticmethod
    def backward(fctx, gx, gv):
        sim = fctx.sim
        (k,) = fctx.saved_tensors
        sim.set_constants(k)
        V = sim.ctx.V
        dev = sim.ctx.device
        gx = torch.zeros((3, V), device=dev) if gx is None else gx.contiguous().float()
        gv = torch.zeros((3, V), device=dev) if gv is None else gv.contiguous().float()
        gk = torch.zeros((sim.ctx.B, 5), dtype=torch.float64, device=dev)
        for seg in reversed(range(len(fctx.starts))):
            x, v = fctx.starts[seg]
            m = min(fctx.every, fctx.n - seg * fctx.every)
            states = [(x, v)]
            for _ in range(m - 1):                       # recompute this segment
                x, v = sim.step(x, v)
                states.append((x, v))
            for j in reversed(range(m)):
                gx, gv, gp = sim.ctx.backward(states[j][0], sim.fields, gx, gv)
                gk += gp
        return gx, gv, gk.to(device=k.device, dtype=k.dtype), None, None, None


def rollout(sim: Simulation, x0, v0, k, n_steps: int, checkpoint_every: int = 10):
    """(x_n, v_n) after n_steps steps from (x0, v0) with constants k [B, 5];
    differentiable in x0, v0 and k."""
    return _Rollout.apply(x0, v0, k, sim, int(n_steps), int(checkpoint_every))


class _Taylor(torch.autograd.Function):
    @staticmethod
    def forward(fctx, x, sim):
        x = x.detach().contiguous()
        fctx.sim = sim
        fctx.save_for_backward(x)
        return sim.ctx.taylor(x)

    @staticmethod
    def backward(fctx, gD):
        (x,) = fctx.saved_tensors
        gx, _ = fctx.sim.ctx.taylor_backward(x, gD)
        return gx, None


def taylor_deformation(sim: Simulation, x):
    """Taylor deformation [B] (float64) of every closed body at x."""
    return _Taylor.apply(x, sim)
