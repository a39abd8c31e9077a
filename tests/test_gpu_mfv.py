"""MFV scheme (moving faces with mass fluxes, O15) on the CUDA path vs the
FP64 oracle through the C ABI: the flux pass on the oracle's frozen H, n and
gradients, one full step, a short rollout, and the properties the scheme
guarantees (pairwise antisymmetry, exact mass bookkeeping, a uniform flow
staying uniform, batching and graph replay).  FP64 within 1e-10 of each
field's RMS (max error), FP32 within 2e-5 (RMS error)."""
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
    return {"sod": I.sod, "turb": I.turbulence, "sedov": I.sedov, "kh": I.kh}[kind](n)


def mfv_ctx(counts, prec):
    m = gz()
    return m.Context(counts if isinstance(counts, list) else [counts],
                     m.default_params(precision=prec, scheme=m.GZ_MFV))


def opar():
    return O.params(scheme=O.MFV)


@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, TOL32)])
@pytest.mark.parametrize("kind,n", [("sod", 23), ("turb", 24), ("sedov", 21)])
def test_mfv_fluxes_vs_oracle(kind, n, prec, tol):
    import torch
    q = cast_state(make(kind, n), prec)
    s = ostate(q)
    p = opar()
    Ho, no, _, _ = O.density(s, p)
    g = O.gradients(s, Ho, no, p)
    grad, B = g["grad"], g["B"]
    if prec == 1:  # the FP32 path reads every input rounded to float
        Ho, no, grad, B = (a.astype(np.float32).astype(np.float64) for a in (Ho, no, grad, B))
    _, dt = O.timestep(s, Ho, no, p)
    cnt = O.Counters()
    dp_o, dE_o, dm_o = O.fluxes(s, Ho, no, grad, B, dt, p, counters=cnt, with_mass=True)
    ctx = mfv_ctx(s.N, prec)
    d = device(q, prec, H=Ho)
    T = d["x"].dtype
    dp, dE, dm = ctx.hydro_fluxes(d, torch.as_tensor(no, dtype=T).cuda(),
                                  torch.as_tensor(grad, dtype=T).cuda().contiguous(),
                                  torch.as_tensor(B, dtype=T).cuda().contiguous(), dt, with_mass=True)
    st = ctx.status(reset=True)
    assert st["ok"], st
    if prec == 0:
        assert st["counters"]["fallback"] == cnt.fallback
        assert st["counters"]["pstar_neg"] == cnt.pstar_neg
    dp, dE, dm = dp.cpu().numpy(), dE.cpu().numpy(), dm.cpu().numpy()
    assert np.abs(dm_o).max() > 0.0
    for name, got, ref in [("dp0", dp[0], dp_o[0]), ("dp1", dp[1], dp_o[1]), ("dp2", dp[2], dp_o[2]),
                           ("dE", dE, dE_o), ("dm", dm, dm_o)]:
        mx, rm = field_err(got, ref)
        assert (mx if prec == 0 else rm) <= tol, (name, mx, rm)


@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, TOL32)])
@pytest.mark.parametrize("kind,n", [("turb", 22), ("sod", 20)])
def test_mfv_full_step_vs_oracle(kind, n, prec, tol):
    import torch
    q = cast_state(make(kind, n), prec)
    s = ostate(q)
    o, dt_o, _, _, _, _ = O.step(s, opar(), with_mass=True)
    ctx = mfv_ctx(s.N, prec)
    d = device(q, prec)
    dtu = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.step(d, 0.0, dtu)
    st = ctx.status(reset=True)
    assert st["ok"], st
    dt_g = float(dtu.cpu()[0])
    assert abs(dt_g - dt_o) / dt_o <= (1e-12 if prec == 0 else 1e-6)
    k_tol = tol * (1 if prec == 0 else 50)
    for k in ("x", "y", "z"):
        before = getattr(s, k)
        mx, rm = field_err(min_image(d[k].cpu().numpy().astype(np.float64) - before),
                           min_image(getattr(o, k) - before))
        assert (mx if prec == 0 else rm) <= k_tol, (k, mx, rm)
    for k in ("vx", "vy", "vz", "u", "m"):
        mx, rm = field_err(d[k].cpu().numpy().astype(np.float64) - getattr(s, k),
                           getattr(o, k) - getattr(s, k))
        assert (mx if prec == 0 else rm) <= k_tol, (k, mx, rm)
    Hg = d["h"].cpu().numpy()
    assert np.max(np.abs(Hg - o.H) / o.H) <= (1e-12 if prec == 0 else 2e-6)


def test_mfv_rollout_fp64_tracks_the_oracle():
    """Eight CFL steps of the Sod tube: the FP64 path stays on the oracle's
    trajectory (every step dt and every field within 1e-9)."""
    m = gz()
    import torch
    q = cast_state(I.sod(14), m.GZ_FP64)
    s = ostate(q)
    ctx = mfv_ctx(s.N, m.GZ_FP64)
    d = device(q, m.GZ_FP64)
    dtu = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(8):
        s, dt_o, _, _, _, _ = O.step(s, opar(), with_mass=True)
        ctx.step(d, 0.0, dtu)
        assert abs(float(dtu.cpu()[0]) - dt_o) <= 1e-9 * dt_o
    st = ctx.status(reset=True)
    assert st["ok"], st
    for k in ("x", "y", "z", "vx", "vy", "vz", "u", "m"):
        g = d[k].cpu().numpy()
        ref = getattr(s, k)
        diff = min_image(g - ref) if k in ("x", "y", "z") else g - ref
        scale = 1.0 if k in ("x", "y", "z") else max(np.sqrt(np.mean(ref * ref)), 1e-300)
        assert np.max(np.abs(diff)) / scale <= 1e-9, (k, np.max(np.abs(diff)) / scale)


@pytest.mark.parametrize("prec", [0, 1])
def test_mfv_pair_contributions_are_bitwise_opposite(prec):
    """Two-particle boxes: both particles get one face's fluxes of mass,
    momentum and energy with exactly opposite signs."""
    import torch
    rng = np.random.default_rng(78)
    T = torch.float64 if prec == 0 else torch.float32
    ctx = mfv_ctx(2, prec)
    nonzero = 0
    for trial in range(40):
        x = rng.uniform(0, 1, (3, 2))
        x[:, 1] = (x[:, 0] + rng.uniform(-0.2, 0.2, 3)) % 1.0
        ids = rng.permutation(2) + int(rng.integers(0, 1000))
        d = {k: torch.as_tensor(v, dtype=T).cuda() for k, v in
             (("x", x[0]), ("y", x[1]), ("z", x[2]), ("vx", rng.normal(0, 1, 2)),
              ("vy", rng.normal(0, 1, 2)), ("vz", rng.normal(0, 1, 2)),
              ("m", rng.uniform(0.5, 2, 2)), ("u", rng.uniform(0.5, 2, 2)),
              ("h", rng.uniform(0.25, 0.45, 2)))}
        d["id"] = torch.as_tensor(ids, dtype=torch.int64).cuda()
        n = torch.as_tensor(rng.uniform(5, 10, 2), dtype=T).cuda()
        grad = torch.as_tensor(rng.normal(0, 0.5, (15, 2)), dtype=T).cuda().contiguous()
        Bm = np.zeros((6, 2))
        Bm[0] = Bm[3] = Bm[5] = rng.uniform(10, 20, 2)
        Bm[1] = rng.uniform(-2, 2, 2)
        B = torch.as_tensor(Bm, dtype=T).cuda().contiguous()
        dp, dE, dm = ctx.hydro_fluxes(d, n, grad, B, float(rng.uniform(0, 0.01)), with_mass=True)
        dp, dE, dm = dp.cpu().numpy(), dE.cpu().numpy(), dm.cpu().numpy()
        assert np.array_equal(dp[:, 0], -dp[:, 1]), (trial, dp)
        assert dE[0] == -dE[1], (trial, dE)
        assert dm[0] == -dm[1], (trial, dm)
        nonzero += dm[0] != 0.0
    assert nonzero > 20
    ctx.status(reset=True)


@pytest.mark.parametrize("prec", [0, 1])
def test_mfv_steps_conserve_mass_and_move_it(prec):
    import torch
    m = gz()
    q = cast_state(I.turbulence(20, seed=11), prec)
    ctx = mfv_ctx(q.N, prec)
    d = device(q, prec)
    m0 = d["m"].double().sum().item()
    for _ in range(5):
        ctx.step(d)
    st = ctx.status(reset=True)
    assert st["ok"], st
    mass = d["m"].double()
    assert abs(mass.sum().item() - m0) <= (1e-13 if prec == 0 else 1e-6) * m0
    assert torch.all(mass > 0)
    rel = (mass.cpu().numpy() - q.m) / q.m
    assert np.abs(rel).max() > 1e-4  # mass moved between particles


@pytest.mark.parametrize("prec", [0, 1])
def test_mfv_uniform_flow_on_a_lattice_has_zero_rates(prec):
    """A uniform state moving with constant velocity on a perfect lattice: every
    face's moving-frame Riemann problem is trivial and the rates cancel."""
    import torch
    n = 10
    x, y, z, _ = I.lattice(n, np.random.default_rng(0), 0.0)
    N = x.size
    q = I.turbulence(n)
    for k, v in (("x", x), ("y", y), ("z", z), ("vx", np.full(N, 0.3)), ("vy", np.full(N, -0.2)),
                 ("vz", np.full(N, 0.1)), ("m", np.full(N, 1.0 / N)), ("u", np.full(N, 1.5)),
                 ("H", np.full(N, I.h0(N)))):
        setattr(q, k, v)
    q = cast_state(q, prec)
    s = ostate(q)
    p = opar()
    Ho, no, _, _ = O.density(s, p)
    g = O.gradients(s, Ho, no, p)
    ctx = mfv_ctx(N, prec)
    d = device(q, prec, H=Ho)
    T = d["x"].dtype
    dp, dE, dm = ctx.hydro_fluxes(d, torch.as_tensor(no, dtype=T).cuda(),
                                  torch.as_tensor(g["grad"], dtype=T).cuda().contiguous(),
                                  torch.as_tensor(g["B"], dtype=T).cuda().contiguous(), 1e-3,
                                  with_mass=True)
    ctx.status(reset=True)
    # scale: one face's mass flux rho |v| |A| with |A| ~ V^(2/3)
    tol = 1e-12 if prec == 0 else 1e-4
    flux_scale = 1.0 * 0.37 * (1.0 / N) ** (2.0 / 3.0)
    assert dm.abs().max().item() <= tol * flux_scale
    assert dp.abs().max().item() <= tol * flux_scale * 2
    assert dE.abs().max().item() <= tol * flux_scale * 3


def test_mfm_context_reports_zero_mass_rates():
    m = gz()
    import torch
    q = cast_state(I.turbulence(12), m.GZ_FP64)
    s = ostate(q)
    Ho, no, _, _ = O.density(s, O.params())
    g = O.gradients(s, Ho, no, O.params())
    ctx = m.Context([s.N], m.default_params(precision=m.GZ_FP64))
    d = device(q, m.GZ_FP64, H=Ho)
    _, _, dm = ctx.hydro_fluxes(d, torch.as_tensor(no).cuda(), torch.as_tensor(g["grad"]).cuda(),
                                torch.as_tensor(g["B"]).cuda(), 1e-3, with_mass=True)
    assert ctx.status(reset=True)["ok"]
    assert torch.count_nonzero(dm).item() == 0
    m0 = d["m"].clone()
    ctx.step(d)
    assert torch.equal(d["m"], m0)


@pytest.mark.parametrize("prec", [0, 1])
def test_mfv_batched_boxes_and_graph_replay_equal_single_steps(prec):
    m = gz()
    import torch
    boxes = [I.sod(9, seed=5), I.sedov(11, seed=6), I.turbulence(10, seed=7)]
    qs = [cast_state(b, prec) for b in boxes]
    off = 0
    for qb in qs:
        qb.id = qb.id + off
        off += qb.N
    singles = []
    for qb in qs:
        ctx = mfv_ctx(qb.N, prec)
        d = device(qb, prec)
        ctx.step(d)
        ctx.step(d)
        singles.append({k: v.cpu().numpy() for k, v in d.items()})
    cat = {k: np.concatenate([getattr(qb, k) for qb in qs]) for k in
           ("x", "y", "z", "vx", "vy", "vz", "m", "u", "H", "id")}
    T = torch.float64 if prec == 0 else torch.float32

    def fresh():
        d = {k: torch.as_tensor(v, dtype=T).cuda() for k, v in cat.items() if k not in ("H", "id")}
        d["h"] = torch.as_tensor(cat["H"], dtype=T).cuda()
        d["id"] = torch.as_tensor(cat["id"], dtype=torch.int64).cuda()
        return d

    counts = [qb.N for qb in qs]
    d1 = fresh()
    ctx = mfv_ctx(counts, prec)
    ctx.step(d1)
    ctx.step(d1)
    assert ctx.status(reset=True)["ok"]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        d2 = fresh()
        ctx2 = m.Context(counts, m.default_params(precision=prec, scheme=m.GZ_MFV), stream=stream)
        ctx2.graph_capture(d2, 2)
        ctx2.graph_launch()
        torch.cuda.synchronize()
    assert ctx2.status(reset=True)["ok"]
    off = 0
    for b, qb in enumerate(qs):
        for k in ("x", "y", "z", "vx", "vy", "vz", "u", "m", "h"):
            got = d1[k].cpu().numpy()[off:off + qb.N]
            assert np.array_equal(got, singles[b][k]), (b, k)
            assert np.array_equal(d2[k].cpu().numpy()[off:off + qb.N], singles[b][k]), (b, k, "graph")
        off += qb.N


def test_adjoint_calls_refuse_mfv():
    m = gz()
    import torch
    q = cast_state(I.turbulence(8), m.GZ_FP64)
    ctx = mfv_ctx(q.N, m.GZ_FP64)
    d = device(q, m.GZ_FP64)
    z = torch.zeros(3, q.N, dtype=torch.float64, device="cuda")
    z1 = torch.zeros(q.N, dtype=torch.float64, device="cuda")
    grad = torch.zeros(15, q.N, dtype=torch.float64, device="cuda")
    B = torch.zeros(6, q.N, dtype=torch.float64, device="cuda")
    with pytest.raises(m.GZError) as e:
        ctx.hydro_fluxes_backward(d, z1 + 1.0, grad, B, 1e-3, z, z1)
    assert e.value.code == 1
    ck = ctx.new_checkpoint(1)
    with pytest.raises(m.GZError) as e:
        ctx.step(d, 1e-4, ckpt=ck, level=1)
    assert e.value.code == 1
    gb = {k: torch.zeros(q.N, dtype=torch.float64, device="cuda") for k in
          ("x", "y", "z", "vx", "vy", "vz", "m", "u", "h")}
    gb["id"] = d["id"]
    gs = {k: torch.zeros_like(v) for k, v in gb.items()}
    with pytest.raises(m.GZError) as e:
        ctx.step_backward(d, 1e-4, gb, gs)
    assert e.value.code == 1
