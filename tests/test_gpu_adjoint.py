"""Hand-written CUDA adjoints vs the derivative oracle (torch autograd of the
step written in plain PyTorch CPU ops), through the C ABI.

Inputs are smooth (no exactly uniform field, which would be a kink of the
limiter).  FP64 path: element-wise within 1e-9 of each adjoint field's RMS.
FP32 path: RMS error within 1e-3 of the FP64 oracle's adjoint (reported)."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import torch_step as TS
from paper_1712_01294_gb300 import inputs as I

from gpu_common import cast_state, device, ostate

pytestmark = pytest.mark.gpu

GAM = 5.0 / 3.0


def gz():
    import paper_1712_01294_gb300 as m
    return m


def rms(a):
    a = np.asarray(a, dtype=np.float64)
    return float(np.sqrt(np.mean(a * a)))


FAILS = []


def check(name, got, ref, prec, tol64=1e-9, tol32=1e-3):
    """Records (not asserts) the error of one adjoint field; see assert_all."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = rms(ref) or 1.0
    rel = np.abs(got - ref) / scale
    err = float(rel.max()) if prec == 0 else rms(got - ref) / scale
    if err > (tol64 if prec == 0 else tol32):
        bad = np.flatnonzero(rel > (tol64 if prec == 0 else tol32))
        FAILS.append((name, err, int(bad.size), bad[:5].tolist(), got[bad[:3]].tolist(),
                      ref[bad[:3]].tolist()))
    return err


def assert_all():
    msg = "\n".join(str(f) for f in FAILS)
    FAILS.clear()
    assert not msg, msg


@pytest.mark.parametrize("prec", [0, 1])
def test_flux_adjoint_matches_autograd(prec):
    m = gz()
    q = cast_state(I.smooth_turbulence(12, seed=3), prec)
    s = ostate(q)
    prm = O.params()
    Ho, no, _, _ = O.density(s, prm)
    g = O.gradients(s, Ho, no, prm)
    grad, B = g["grad"], g["B"]
    if prec == m.GZ_MIXED32:
        Ho, no, grad, B = (a.astype(np.float32).astype(np.float64) for a in (Ho, no, grad, B))
    _, dt = O.timestep(s, Ho, no, prm)
    poff, pnb = O.flux_pairs(s, Ho)
    L, R = TS.canonical_pairs(poff, pnb, s.id)
    rng = np.random.default_rng(5)
    dpbar = rng.normal(size=(3, s.N))
    dEbar = rng.normal(size=s.N)
    # oracle: autograd of the flux stage with every input a leaf
    T = lambda a: torch.tensor(np.asarray(a, dtype=np.float64), requires_grad=True)
    x, y, z = T(s.x), T(s.y), T(s.z)
    rho0 = s.m * no
    if prec == m.GZ_MIXED32:
        rho0 = (s.m.astype(np.float32) * no.astype(np.float32)).astype(np.float64)
        P0 = ((np.float32(GAM - 1.0) * rho0.astype(np.float32)) * s.u.astype(np.float32)).astype(np.float64)
    else:
        P0 = (GAM - 1.0) * rho0 * s.u
    prim = [T(rho0), T(s.vx), T(s.vy), T(s.vz), T(P0)]
    H, n = T(Ho), T(no)
    gl_leaves = [T(grad[k]) for k in range(15)]
    gl = [[gl_leaves[3 * f + k] for k in range(3)] for f in range(5)]
    Bl = [T(B[k]) for k in range(6)]
    dp, dE = TS.flux_stage(x, y, z, prim, H, n, gl, Bl, L, R, dt)
    J = sum((dp[k] * torch.tensor(dpbar[k])).sum() for k in range(3)) + (dE * torch.tensor(dEbar)).sum()
    leaves = [x, y, z] + prim + [H, n] + gl_leaves + Bl
    ref = [t.numpy() for t in torch.autograd.grad(J, leaves, allow_unused=True)]
    # CUDA adjoint
    ctx = m.Context([s.N], m.default_params(precision=prec))
    d = device(q, prec, H=Ho)
    Tt = d["x"].dtype
    out = ctx.hydro_fluxes_backward(d, torch.as_tensor(no, dtype=Tt).cuda(),
                                    torch.as_tensor(grad, dtype=Tt).cuda().contiguous(),
                                    torch.as_tensor(B, dtype=Tt).cuda().contiguous(), dt,
                                    torch.as_tensor(dpbar).cuda().contiguous(),
                                    torch.as_tensor(dEbar).cuda().contiguous())
    st = ctx.status(reset=True)
    assert st["ok"], st
    o = {k: v.cpu().numpy() for k, v in out.items()}
    errs = {}
    for k in range(3):
        errs[f"x{k}"] = check(f"x{k}", o["x"][k], ref[k], prec)
    for f in range(5):
        errs[f"W{f}"] = check(f"W{f}", o["W"][f], ref[3 + f], prec)
    errs["H"] = check("H", o["h"], ref[8], prec)
    errs["n"] = check("n", o["n"], ref[9], prec)
    for q_ in range(15):
        errs[f"g{q_}"] = check(f"g{q_}", o["grad"][q_], ref[10 + q_], prec)
    for q_ in range(6):
        errs[f"B{q_}"] = check(f"B{q_}", o["B"][q_], ref[25 + q_], prec)
    print("flux adjoint errors", prec, {k: f"{v:.2e}" for k, v in errs.items()})
    assert_all()


KEYS = ("x", "y", "z", "vx", "vy", "vz", "m", "u")
OUTK = ("x", "y", "z", "vx", "vy", "vz", "u")


def step_adjoint_case(make, prec, seed=7, tol=None):
    """(oracle gradient dict, CUDA gradient dict) of J = sum <gbar, state_after>
    with respect to the state before one step (dt and neighbour sets frozen)."""
    m = gz()
    q = cast_state(make(), prec)
    prm = O.params(tol=1e-12 if prec == 0 else 1e-6)
    fr, s, Hs, n = TS.freeze(q.__dict__, prm)
    st = TS.as_tensors(s, requires_grad=True)
    out = TS.step(st, fr)
    rng = np.random.default_rng(seed)
    gbar = {k: rng.normal(size=s.N) for k in OUTK}
    J = sum((out[k] * torch.tensor(gbar[k])).sum() for k in OUTK)
    ref = dict(zip(KEYS, (g.numpy() for g in torch.autograd.grad(J, [st[k] for k in KEYS]))))
    ctx = m.Context([s.N], m.default_params(precision=prec, tol=1e-12 if prec == 0 else 1e-6))
    d = device(q, prec)
    T = d["x"].dtype
    gend = {k: torch.as_tensor(gbar[k], dtype=T).cuda().contiguous() for k in OUTK}
    gstart = {k: torch.zeros(s.N, dtype=T, device="cuda") for k in KEYS}
    ctx.step_backward(d, fr.dt, gend, gstart)
    st_ = ctx.status(reset=True)
    assert st_["ok"], st_
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in gstart.items()}
    return ref, got


@pytest.mark.parametrize("prec", [0, 1])
def test_step_adjoint_matches_autograd(prec):
    ref, got = step_adjoint_case(lambda: I.smooth_turbulence(12, seed=3), prec)
    errs = {k: check(k, got[k], ref[k], prec) for k in KEYS}
    print("step adjoint errors", prec, {k: f"{v:.2e}" for k, v in errs.items()})
    assert_all()
