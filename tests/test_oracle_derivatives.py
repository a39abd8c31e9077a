"""Pins of the derivative oracle (oracle/torch_step.py, the step written in
plain PyTorch CPU ops): its forward step equals the C oracle's, and its
dual-number (forward-mode) directional derivatives equal central finite
differences of the C oracle on smooth inputs."""
import numpy as np
import pytest
import torch
import torch.autograd.forward_ad as fwAD

import oracle as O
from oracle import torch_step as TS
from paper_1712_01294_gb300 import inputs as I

KEYS = ("x", "y", "z", "vx", "vy", "vz", "m", "u")
OUTK = ("x", "y", "z", "vx", "vy", "vz", "u")
PRM = O.params(tol=1e-12)


@pytest.mark.parametrize("make", [lambda: I.kh(10, seed=3), lambda: I.turbulence(10, seed=4),
                                  lambda: I.sedov(9, seed=5)])
def test_torch_step_equals_c_oracle_step(make):
    p = make()
    fr, s, Hs, n = TS.freeze(p.__dict__, PRM)
    out = TS.step(TS.as_tensors(s), fr, return_all=True)
    o, dt, n_o, dp_o, dE_o = O.step(s, PRM, dt=fr.dt)
    for k in OUTK:
        a, b = out[k].numpy(), getattr(o, k)
        assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.abs(b).max()), k
    assert np.max(np.abs(out["dpdt"].numpy() - dp_o)) <= 1e-11 * np.abs(dp_o).max()
    assert np.max(np.abs(out["dEdt"].numpy() - dE_o)) <= 1e-11 * np.abs(dE_o).max()
    assert np.max(np.abs(out["H"].numpy() - o.H) / o.H) <= 1e-12


def _fd(s, fr, gbar, delta, eps):
    def run(e):
        q = s.copy()
        for k in KEYS:
            setattr(q, k, getattr(s, k) + e * delta[k].numpy())
        for k in ("x", "y", "z"):
            v = getattr(q, k)
            setattr(q, k, np.where(v < 0, v + 1, np.where(v >= 1, v - 1, v)))
        return O.step(q, PRM, dt=fr.dt)[0]
    op, om = run(eps), run(-eps)
    tot = 0.0
    for k in OUTK:
        d = getattr(op, k) - getattr(om, k)
        if k in ("x", "y", "z"):
            d = np.where(d > 0.5, d - 1, np.where(d < -0.5, d + 1, d))
        tot += float(np.sum(d * gbar[k].numpy()))
    return tot / (2 * eps)


@pytest.mark.parametrize("make", [lambda: I.smooth_turbulence(10, seed=5),
                                  lambda: I.smooth_turbulence(9, seed=11)])
def test_dual_number_derivative_matches_finite_differences(make):
    p = make()
    fr, s, _, _ = TS.freeze(p.__dict__, PRM)
    st = TS.as_tensors(s)
    rng = np.random.default_rng(1)
    gbar = {k: torch.tensor(rng.normal(size=s.N)) for k in OUTK}
    scale = {"x": 0.1, "y": 0.1, "z": 0.1, "vx": 1.0, "vy": 1.0, "vz": 1.0, "m": s.m.mean(), "u": 1.0}
    for var in KEYS:
        delta = {k: torch.zeros(s.N, dtype=torch.float64) for k in KEYS}
        delta[var] = torch.tensor(rng.normal(size=s.N) * scale[var])
        with fwAD.dual_level():
            out = TS.step({k: fwAD.make_dual(st[k], delta[k]) for k in KEYS}, fr)
            J = sum((out[k] * gbar[k]).sum() for k in OUTK)
            ad = fwAD.unpack_dual(J).tangent.item()
        fd = _fd(s, fr, gbar, delta, 1e-6)
        # a dropped term or sign is an O(1) error; 2e-5 leaves room for the rare
        # neighbour crossing the support edge inside the finite-difference step
        assert abs(ad - fd) <= 2e-5 * abs(fd) + 1e-9, (var, ad, fd)


def test_reverse_gradient_agrees_with_dual_numbers():
    p = I.smooth_turbulence(8, seed=7)
    fr, s, _, _ = TS.freeze(p.__dict__, PRM)
    rng = np.random.default_rng(2)
    gbar = {k: torch.tensor(rng.normal(size=s.N)) for k in OUTK}
    delta = {k: torch.tensor(rng.normal(size=s.N)) for k in KEYS}
    st = TS.as_tensors(s, requires_grad=True)
    out = TS.step(st, fr)
    J = sum((out[k] * gbar[k]).sum() for k in OUTK)
    g = torch.autograd.grad(J, [st[k] for k in KEYS])
    rev = sum(float((gi * delta[k]).sum()) for gi, k in zip(g, KEYS))
    with fwAD.dual_level():
        st0 = TS.as_tensors(s)
        out = TS.step({k: fwAD.make_dual(st0[k], delta[k]) for k in KEYS}, fr)
        J = sum((out[k] * gbar[k]).sum() for k in OUTK)
        ad = fwAD.unpack_dual(J).tangent.item()
    assert abs(rev - ad) <= 1e-12 * abs(ad)
