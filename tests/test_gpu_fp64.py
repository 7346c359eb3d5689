"""The float64 MLS option (ibm_interpolate_fp64: the general 4x4 moment
system of Eqs. mls_A..mls_Q solved by LU, face geometry in float64) against
the FP64 oracle, beside the float32 closed form of the marker kernels.

The float64 path differs from the oracle only by the float32 storage of its
outputs (half an ulp per element, rel. L2 <= 2^-24 ~ 6e-8); the closed form
in float32 carries float32 arithmetic on top (bar 1e-5)."""
import numpy as np
import pytest
import torch

from oracle import ibm_oracle as O
from paper_1612_03399_gb300 import _lib

import helpers as H
from test_gpu_parity import mixed_workload, tie_free_state

pytestmark = pytest.mark.gpu
DEV = "cuda"


def test_fp64_interpolation_matches_oracle_to_storage(record_error):
    wl = mixed_workload()
    ob = H.oracle_bodies(wl)
    ctx = _lib.Context(wl.bodies, wl.grid, dt=wl.dt, mu=wl.mu, alpha=wl.alpha)
    rel = tie_free_state(wl, 50, scale=0.03, stretch=0.03)
    x = H.state_tensor(wl, rel)
    xs = H.to_abs(wl, H.split_state(ctx, wl, x))
    rng = np.random.default_rng(51)
    v = torch.tensor(rng.uniform(-0.5, 0.5, (3, ctx.V)), dtype=torch.float32, device=DEV)
    fields = H.fields_for(wl, DEV)
    U64, Fm64, Fe64 = ctx.interpolate_fp64(x, v, fields)
    U32, Fm32, Fe32 = ctx.interpolate(x, v, fields)
    ctx.check_device_error()
    vs = [torch.tensor(a) for a in H.split_state(ctx, wl, v)]
    out = O.step(ob, xs, vs, tuple(f.double().cpu() for f in fields), H.oracle_params(wl),
                 with_spread=False)
    for name, g64, g32 in (("U", U64, U32), ("F_marker", Fm64, Fm32), ("F_ext_face", Fe64, Fe32)):
        ref = out[name].numpy()
        e64 = H.rel_l2(g64.double().cpu().numpy().T, ref)
        e32 = H.rel_l2(g32.double().cpu().numpy().T, ref)
        record_error(f"{name}_fp64", e64)
        record_error(f"{name}_fp32", e32)
        assert e64 <= 1e-7, (name, e64)
        assert e32 <= 1e-5, (name, e32)
