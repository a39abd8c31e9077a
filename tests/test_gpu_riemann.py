"""Riemann-solver option of the MFM face on the CUDA path vs the FP64 oracle
(exact star on every face, or HLLC with the exact star where HLLC's P* < 0):
the flux pass on the oracle's frozen H, n and gradients, one full step, and
the pair antisymmetry.  FP64 within 1e-10 of each field's RMS (max error),
FP32 within 2e-5 (RMS error)."""
import numpy as np
import pytest

import oracle as O
from paper_1712_01294_gb300 import inputs as I

from gpu_common import cast_state, device, field_err, min_image, ostate

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 2e-5


def gz():
    import paper_1712_01294_gb300 as m
    return m


def make(kind, n):
    if kind == "r123":  # strong double rarefaction: HLLC's P* < 0 on many faces
        return I.sod(n, rho_l=1.0, p_l=0.4, rho_r=1.0, p_r=0.4, u_l=-2.0, u_r=2.0)
    return {"sod": I.sod, "turb": I.turbulence, "sedov": I.sedov}[kind](n)


def ctx_for(N, prec, riemann):
    m = gz()
    return m.Context([N], m.default_params(precision=prec, riemann=riemann))


@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, TOL32)])
@pytest.mark.parametrize("riemann", [1, 2])
@pytest.mark.parametrize("kind,n", [("turb", 19), ("r123", 17), ("sedov", 16)])
def test_riemann_option_fluxes_vs_oracle(kind, n, riemann, prec, tol):
    import torch
    q = cast_state(make(kind, n), prec)
    s = ostate(q)
    p = O.params(riemann=riemann)
    Ho, no, _, _ = O.density(s, p)
    g = O.gradients(s, Ho, no, p)
    grad, B = g["grad"], g["B"]
    if prec == 1:
        Ho, no, grad, B = (a.astype(np.float32).astype(np.float64) for a in (Ho, no, grad, B))
    _, dt = O.timestep(s, Ho, no, p)
    cnt = O.Counters()
    dp_o, dE_o = O.fluxes(s, Ho, no, grad, B, dt, p, counters=cnt)
    ctx = ctx_for(s.N, prec, riemann)
    d = device(q, prec, H=Ho)
    T = d["x"].dtype
    dp, dE = ctx.hydro_fluxes(d, torch.as_tensor(no, dtype=T).cuda(),
                              torch.as_tensor(grad, dtype=T).cuda().contiguous(),
                              torch.as_tensor(B, dtype=T).cuda().contiguous(), dt)
    st = ctx.status(reset=True)
    assert st["ok"], st
    if prec == 0:
        assert st["counters"]["pstar_neg"] == cnt.pstar_neg
        assert st["counters"]["fallback"] == cnt.fallback
    if kind == "r123" and riemann == 2:  # faces the fallback repaired
        assert cnt.pstar_neg > 0
    dp, dE = dp.cpu().numpy(), dE.cpu().numpy()
    for name, got, ref in [("dp0", dp[0], dp_o[0]), ("dp1", dp[1], dp_o[1]), ("dp2", dp[2], dp_o[2]),
                           ("dE", dE, dE_o)]:
        mx, rm = field_err(got, ref)
        assert (mx if prec == 0 else rm) <= tol, (name, mx, rm)


@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, TOL32)])
@pytest.mark.parametrize("riemann", [1, 2])
def test_riemann_option_full_step_vs_oracle(riemann, prec, tol):
    import torch
    q = cast_state(make("r123", 16), prec)
    s = ostate(q)
    o, dt_o, _, _, _ = O.step(s, O.params(riemann=riemann))
    ctx = ctx_for(s.N, prec, riemann)
    d = device(q, prec)
    dtu = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.step(d, 0.0, dtu)
    st = ctx.status(reset=True)
    assert st["ok"], st
    assert abs(float(dtu.cpu()[0]) - dt_o) / dt_o <= (1e-12 if prec == 0 else 1e-6)
    k_tol = tol * (1 if prec == 0 else 50)
    for k in ("x", "y", "z"):
        before = getattr(s, k)
        mx, rm = field_err(min_image(d[k].cpu().numpy().astype(np.float64) - before),
                           min_image(getattr(o, k) - before))
        assert (mx if prec == 0 else rm) <= k_tol, (k, mx, rm)
    for k in ("vx", "vy", "vz", "u"):
        mx, rm = field_err(d[k].cpu().numpy().astype(np.float64) - getattr(s, k),
                           getattr(o, k) - getattr(s, k))
        assert (mx if prec == 0 else rm) <= k_tol, (k, mx, rm)


@pytest.mark.parametrize("prec", [0, 1])
def test_exact_pair_contributions_are_bitwise_opposite(prec):
    import torch
    rng = np.random.default_rng(79)
    T = torch.float64 if prec == 0 else torch.float32
    ctx = ctx_for(2, prec, 1)
    for trial in range(30):
        x = rng.uniform(0, 1, (3, 2))
        x[:, 1] = (x[:, 0] + rng.uniform(-0.2, 0.2, 3)) % 1.0
        ids = rng.permutation(2) + int(rng.integers(0, 1000))
        d = {k: torch.as_tensor(v, dtype=T).cuda() for k, v in
             (("x", x[0]), ("y", x[1]), ("z", x[2]), ("vx", rng.normal(0, 1.5, 2)),
              ("vy", rng.normal(0, 1.5, 2)), ("vz", rng.normal(0, 1.5, 2)),
              ("m", rng.uniform(0.5, 2, 2)), ("u", rng.uniform(0.5, 2, 2)),
              ("h", rng.uniform(0.25, 0.45, 2)))}
        d["id"] = torch.as_tensor(ids, dtype=torch.int64).cuda()
        n = torch.as_tensor(rng.uniform(5, 10, 2), dtype=T).cuda()
        grad = torch.as_tensor(rng.normal(0, 0.5, (15, 2)), dtype=T).cuda().contiguous()
        Bm = np.zeros((6, 2))
        Bm[0] = Bm[3] = Bm[5] = rng.uniform(10, 20, 2)
        B = torch.as_tensor(Bm, dtype=T).cuda().contiguous()
        dp, dE = ctx.hydro_fluxes(d, n, grad, B, float(rng.uniform(0, 0.01)))
        dp, dE = dp.cpu().numpy(), dE.cpu().numpy()
        assert np.array_equal(dp[:, 0], -dp[:, 1]), (trial, dp)
        assert dE[0] == -dE[1], (trial, dE)
    ctx.status(reset=True)


def test_invalid_riemann_combinations_are_refused():
    m = gz()
    import torch
    with pytest.raises(m.GZError):
        m.Context([64], m.default_params(scheme=m.GZ_MFV, riemann=m.GZ_RIEMANN_EXACT))
    with pytest.raises(m.GZError):
        m.Context([64], m.default_params(riemann=3))
    q = cast_state(I.turbulence(8), m.GZ_FP64)
    ctx = ctx_for(q.N, m.GZ_FP64, m.GZ_RIEMANN_FALLBACK)
    d = device(q, m.GZ_FP64)
    ck = ctx.new_checkpoint(1)
    with pytest.raises(m.GZError) as e:
        ctx.step(d, 1e-4, ckpt=ck, level=1)
    assert e.value.code == 1
