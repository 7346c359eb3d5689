"""Pins of the oracle's strong-coupling integrator, Hamming's fourth-order
predictor-corrector with a Runge-Kutta start (reading R19); no GPU.

The global error must fall at least as h^4 (the final 9/121 correction
removes the leading local error term, so smooth problems show up to h^5);
a wrong coefficient anywhere drops the order to 2 or below."""
import math

import numpy as np
import pytest
import torch

from oracle import ibm_oracle as O
from paper_1612_03399_gb300 import workloads as W

DT = torch.float64


def run(f, y0, h, t_end):
    H = O.Hamming(f, y0, h)
    y = y0
    for _ in range(int(round(t_end / h))):
        y = H.step()
    return y


def orders(errors):
    return [math.log2(a / b) for a, b in zip(errors, errors[1:])]


def test_fourth_order_on_a_decaying_exponential():
    lam = -1.3
    f = lambda y: lam * y
    y0 = torch.tensor([1.0], dtype=DT)
    errs = [abs(float(run(f, y0, h, 1.0)) - math.exp(lam)) for h in (0.05, 0.025, 0.0125)]
    assert all(3.6 < p < 6.5 for p in orders(errs)), orders(errs)


def test_fourth_order_on_a_harmonic_oscillator():
    w = 2.0
    f = lambda y: torch.stack([y[1], -w * w * y[0]])
    y0 = torch.tensor([1.0, 0.0], dtype=DT)
    T = 1.0
    exact = torch.tensor([math.cos(w * T), -w * math.sin(w * T)], dtype=DT)
    errs = [float((run(f, y0, h, T) - exact).norm()) for h in (0.04, 0.02, 0.01)]
    assert all(3.6 < p < 6.5 for p in orders(errs)), orders(errs)


def test_exact_for_uniformly_accelerated_motion():
    g = torch.tensor([0.3, -9.8, 1.2], dtype=DT)
    f = lambda y: torch.stack([y[1], g.expand_as(y[1])])
    y0 = torch.stack([torch.tensor([[0.1, 0.2, 0.3]], dtype=DT), torch.tensor([[1.0, 0.5, -2.0]], dtype=DT)])
    h, n = 0.01, 25
    H = O.Hamming(f, y0, h)
    for _ in range(n):
        y = H.step()
    t = n * h
    x_exact = y0[0] + y0[1] * t + 0.5 * g * t * t
    assert torch.allclose(y[0], x_exact, rtol=0, atol=1e-14)
    assert torch.allclose(y[1], y0[1] + g * t, rtol=0, atol=1e-13)


def test_fourth_order_on_a_drop_in_shear():
    """The mesh problem itself (springs, bending, area, volume and the probe
    traction in a linear shear): positions after a fixed time converge at
    fourth order against a run with a four times smaller step."""
    v, t = W.icosphere(2)
    c = np.array([0.5, 0.5, 0.5])
    b = O.Body(c + 0.2 * v, t, c, ks=1.0, kb=0.05, ka=1.0, kA=1.0, kv=1.0)
    n = (24, 24, 24)
    fields = tuple(f.to(DT) for f in W.sample_field({"kind": "shear"}, W.Grid(n), dtype=torch.float64))
    rng = np.random.default_rng(0)
    x0 = torch.tensor(c + 0.2 * v * (1.0 + 0.02 * rng.standard_normal((len(v), 1))), dtype=DT)
    v0 = torch.zeros_like(x0)
    T = 0.24

    def final(dt):
        prm = O.Params(n, dt=dt)
        return O.hamming_rollout([b], [x0], [v0], fields, prm, int(round(T / dt)))[-1][0][0]

    ref = final(0.0025)
    errs = [float((final(dt) - ref).norm()) for dt in (0.02, 0.01)]
    assert 3.6 < orders(errs)[0] < 6.5, (errs, orders(errs))
