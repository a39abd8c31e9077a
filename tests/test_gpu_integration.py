"""Whole-run checks at the sizes of the workloads the hot path is built for,
through the C ABI: the Sod tube against its exact solution and the oracle,
the Sedov-Taylor blast against its self-similar shock radius, the
Kelvin-Helmholtz differentiable rollout against finite differences, and long
runs (conservation over 400 turbulent steps, 200 ensemble steps without a
status bit)."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_1712_01294_gb300 import inputs as I

from gpu_common import cast_state, device, field_err, ostate

pytestmark = pytest.mark.gpu
GAM = 5.0 / 3.0


def gz():
    import paper_1712_01294_gb300 as m
    return m


# ------------------------------------------------------------------ Sod
def sod_exact_rho(x, t, g=GAM):
    """Exact density of the periodic Sod tube: the split at x = 1/2 (L | R)
    and its mirror at x = 0 (R | L), before their waves meet."""
    A = O.riemann_sample(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, g, (x - 0.5) / t)
    xb = np.where(x >= 0.75, x - 1.0, x)
    B = O.riemann_sample(0.125, 0.0, 0.1, 1.0, 0.0, 1.0, g, xb / t)
    mid = (x >= 0.25) & (x < 0.75)
    return np.where(mid, A[0], B[0])


def binned_rho(ctx, d, n):
    nn, _ = ctx.density(d)
    rho = (d["m"] * nn).double().cpu().numpy()
    x = d["x"].double().cpu().numpy()
    bins = np.minimum((x * n).astype(int), n - 1)
    return np.bincount(bins, rho, n) / np.bincount(bins, None, n)


def test_sod_50_steps_fp64_against_exact_solution_and_oracle():
    """32^3 Sod tube, FP64 path, 50 steps of dt = 0.002 to t = 0.1 (before
    the waves of the two interfaces meet): binned density against the exact
    solution, and every field against the oracle run with the same steps."""
    m = gz()
    q = cast_state(I.sod(32), m.GZ_FP64)
    ctx = m.Context([q.N], m.default_params(precision=m.GZ_FP64))
    d = device(q, m.GZ_FP64)
    dt, nsteps, n = 0.002, 50, 32
    # the fixed step stays inside the CFL limit throughout
    dtu = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(nsteps):
        ctx.step(d, dt, dtu)
    st = ctx.status(reset=True)
    assert st["ok"], st
    rb = binned_rho(ctx, d, n)
    xf = (np.arange(n)[:, None] + (np.arange(16) + 0.5)[None, :] / 16) / n
    ex = sod_exact_rho(xf.ravel(), dt * nsteps).reshape(n, 16).mean(1)
    l1 = float(np.mean(np.abs(rb - ex)))
    print("sod L1(rho) at t = 0.1:", l1)
    assert l1 < 0.09  # the oracle's own 32^3 error is 0.071
    s = ostate(q)
    p = O.params()
    for _ in range(nsteps):
        s, _, _, _, _ = O.step(s, p, dt=dt)
    for k in ("x", "y", "z", "vx", "vy", "vz", "u"):
        mx, rm = field_err(d[k].cpu().numpy(), getattr(s, k))
        print("sod 50-step", k, mx, rm)
        assert rm <= 1e-8, (k, mx, rm)


# ------------------------------------------------------------------ Sedov
def sedov_run(m, prec, n, t_end):
    q = cast_state(I.sedov(n), prec)
    ctx = m.Context([q.N], m.default_params(precision=prec))
    d = device(q, prec)
    dtu = torch.zeros(1, dtype=torch.float64, device="cuda")
    t, steps = 0.0, 0
    while t < t_end and steps < 5000:
        ctx.step(d, 0.0, dtu)
        t += float(dtu.item())
        steps += 1
    st = ctx.status(reset=True)
    assert st["ok"], st
    return ctx, d, t, steps


def shock_radius_measured(ctx, d, nb=100):
    """Radius of the peak of the shell-averaged density about the centre."""
    nn, _ = ctx.density(d)
    rho = (d["m"] * nn).double().cpu().numpy()
    r = np.sqrt(sum((d[k].double().cpu().numpy() - 0.5) ** 2 for k in ("x", "y", "z")))
    keep = r < 0.5
    bins = np.minimum((r[keep] / 0.5 * nb).astype(int), nb - 1)
    prof = np.bincount(bins, rho[keep], nb) / np.maximum(np.bincount(bins, None, nb), 1)
    k = int(np.argmax(prof))
    return (k + 0.5) * 0.5 / nb, float(prof[k])


@pytest.mark.parametrize("prec", [0, 1])
def test_sedov_64cubed_shock_radius_against_self_similar_solution(prec):
    sedov_exact = pytest.importorskip("sedov_exact")
    m = gz()
    ctx, d, t, steps = sedov_run(m, prec, 64, 0.05)
    R, peak = shock_radius_measured(ctx, d)
    Rx = sedov_exact.shock_radius(t)
    print(f"sedov 64^3 prec {prec}: t = {t:.5f} after {steps} steps, R = {R:.4f} vs {Rx:.4f} "
          f"(rel {R / Rx - 1:+.4f}), peak rho {peak:.3f}")
    assert abs(R / Rx - 1.0) < 0.05
    assert peak > 2.0  # a compressed shell (4 for an unresolved strong shock)


def test_sedov_steps_fp32_and_fp64_against_oracle():
    """32^3 blast, five CFL steps: FP64 path within 1e-10 of each field's RMS
    of the oracle run with the same steps, FP32 path within 2e-5 (RMS)."""
    m = gz()
    for prec in (m.GZ_FP64, m.GZ_MIXED32):
        q = cast_state(I.sedov(32), prec)
        ctx = m.Context([q.N], m.default_params(precision=prec))
        d = device(q, prec)
        s = ostate(q)
        p = O.params()
        dtu = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(5):
            ctx.step(d, 0.0, dtu)
            s, _, _, _, _ = O.step(s, p, dt=float(dtu.item()))
        st = ctx.status(reset=True)
        assert st["ok"], st
        for k in ("x", "y", "z", "vx", "vy", "vz", "u"):
            mx, rm = field_err(d[k].cpu().numpy(), getattr(s, k))
            print("sedov 5-step", prec, k, mx, rm)
            assert (mx <= 1e-10) if prec == m.GZ_FP64 else (rm <= 2e-5), (prec, k, mx, rm)


# ------------------------------------------------------------------ KH rollout
def region_ke(state, mask):
    v2 = state["vx"] ** 2 + state["vy"] ** 2 + state["vz"] ** 2
    return (0.5 * state["m"].to(torch.float64) * v2.to(torch.float64) * mask).sum()


def kh_grad(m, prec, q, nsteps, dts=None):
    from paper_1712_01294_gb300 import autograd as GA
    ctx = m.Context([q.N], m.default_params(precision=prec, tol=1e-12 if prec == 0 else 1e-6))
    d = device(q, prec)
    for k in ("vx", "vy", "vz", "u"):
        d[k].requires_grad_(True)
    mask = torch.as_tensor(q.y > 0.75, dtype=torch.float64).cuda()
    fin, used = GA.rollout(ctx, dict(d), nsteps, dts)
    L = region_ke(fin, mask)
    L.backward()
    g = {k: d[k].grad.detach().double().cpu().numpy() for k in ("vx", "vy", "vz", "u")}
    st = ctx.status(reset=True)
    assert st["ok"], st
    return ctx, mask, used, float(L), g


def test_kh_64cubed_10_step_rollout_gradient():
    """The differentiable-rollout workload at its size: 64^3 particles, 10
    steps, loss = kinetic energy of the particles starting at y > 0.75.
    Smooth (tanh) interfaces keep the loss differentiable.  FP64 adjoint
    against central differences of the FP64 forward along the gradient
    (bar 1e-4), and the FP32 adjoint against the FP64 one."""
    m = gz()
    q = I.kh(64, smooth=0.05)
    q64 = cast_state(q, m.GZ_FP64)
    ctx, mask, dts, L0, g64 = kh_grad(m, m.GZ_FP64, q64, 10)
    norm = math.sqrt(sum(float(np.sum(v * v)) for v in g64.values()))
    delta = {k: v / norm for k, v in g64.items()}
    dd = norm  # <g, g / |g|>

    def loss(eps):
        d = device(q64, m.GZ_FP64)
        for k in delta:
            d[k] = d[k] + eps * torch.as_tensor(delta[k]).cuda()
        for dt in dts:
            ctx.step(d, dt)
        return float(region_ke(d, mask))
    fds = [(loss(e) - loss(-e)) / (2 * e) for e in (1e-4, 1e-5, 1e-6)]
    rel = min(abs(fd - dd) / abs(fd) for fd in fds)
    print("kh 64^3 FD", dd, fds, rel)
    assert rel < 1e-4
    q32 = cast_state(q, m.GZ_MIXED32)
    _, _, _, L32, g32 = kh_grad(m, m.GZ_MIXED32, q32, 10, dts)
    errs = {k: float(np.linalg.norm(g32[k] - g64[k]) / np.linalg.norm(g64[k])) for k in g64}
    print("kh 64^3 FP32 vs FP64 adjoint", errs, "loss", L32, L0)
    assert max(errs.values()) < 1e-2
    assert abs(L32 / L0 - 1.0) < 1e-4


def test_kh_64cubed_sharp_layer_rollout_is_deterministic():
    """The workload as specified (sharp layer, FP32, 10 CFL steps): the
    adjoint runs without a device error and gives bitwise the same gradient
    on a second run."""
    m = gz()
    q = cast_state(I.kh(64), m.GZ_MIXED32)
    _, _, dts, L1, g1 = kh_grad(m, m.GZ_MIXED32, q, 10)
    _, _, _, L2, g2 = kh_grad(m, m.GZ_MIXED32, q, 10, dts)
    assert L1 == L2
    for k in g1:
        assert np.all(np.isfinite(g1[k]))
        assert np.array_equal(g1[k], g2[k]), k


def test_kh_64cubed_sharp_layer_fp32_gradient():
    """The workload as specified (sharp layer, 10 FP32 steps, loss = kinetic
    energy of the particles starting at y > 0.75).
    (1) The FP32 adjoint against the FP64 adjoint of the same sharp-layer
        rollout (same steps).
    (2) FP64 central differences.  The sharp layer's vx, rho and P are
        exactly uniform in each region, so at the start every bulk particle
        sits on a limiter kink (0/0 in alpha, tied extremes, degenerate clamp
        bounds), where the step has one-sided derivatives only: along the
        full gradient the limiter's choices change at every eps (about 3.6e5
        of them at eps = 1e-8 as at 1e-5) and central differences differ from
        the adjoint by 1.2e-4.  Along the gradient's vy part (vy is the one
        smooth field; the uniform fields stay uniform at the start) the
        step is smooth at the base point: the limiter's choices that change
        (gz_checkpoint_limiters: limiting neighbour and extreme particle per
        field, every step, at +eps and -eps against the base run) are kinks
        the perturbed runs cross, their number falls with eps, and the
        differences converge to the adjoint."""
    m = gz()
    q = I.kh(64)
    q64 = cast_state(q, m.GZ_FP64)
    ctx64, mask, dts, L64, g64 = kh_grad(m, m.GZ_FP64, q64, 10)
    q32 = cast_state(q, m.GZ_MIXED32)
    _, _, _, L32, g32 = kh_grad(m, m.GZ_MIXED32, q32, 10, dts)
    errs = {k: float(np.linalg.norm(g32[k] - g64[k]) / np.linalg.norm(g64[k])) for k in g64}
    print("kh sharp 64^3: FP32 vs FP64 adjoint", errs, "loss", L32, L64)
    assert abs(L32 / L64 - 1.0) < 1e-4
    assert max(errs.values()) < 2e-2
    ck = ctx64.new_checkpoint(m.GZ_CKPT_GRADIENTS)

    def run(delta, eps):
        d = device(q64, m.GZ_FP64)
        for k in delta:
            d[k] = d[k] + eps * delta[k]
        lims = []
        for dt in dts:
            ctx64.step(d, dt, None, ck, m.GZ_CKPT_GRADIENTS)
            lims.append(ctx64.checkpoint_limiters(ck))
        return float(region_ke(d, mask)), lims

    def fd_rows(delta, epss):
        L0, base = run(delta, 0.0)
        assert abs(L0 / L64 - 1.0) < 1e-12
        rows = []
        for eps in epss:
            Lp, lp = run(delta, eps)
            Lm, lm = run(delta, -eps)
            sw = sum(int((a != b).sum()) + int((c != b).sum()) for a, c, b in zip(lp, lm, base))
            rows.append((eps, sw, (Lp - Lm) / (2 * eps)))
        return rows

    nvy = float(np.linalg.norm(g64["vy"]))
    rows = fd_rows({"vy": torch.as_tensor(g64["vy"] / nvy).cuda()}, (1e-5, 1e-6, 1e-7))
    rel = [(e, sw, abs(fd - nvy) / abs(fd)) for e, sw, fd in rows]
    choices = 2 * 10 * q.N * len(dts)  # both perturbed runs, 10 per particle, every step
    print("kh sharp 64^3 FD along the gradient's vy part (eps, limiter switches, rel to adjoint):",
          rel, "adjoint", nvy, "choices", choices)
    assert rel[0][1] > rel[1][1] > rel[2][1]   # crossings made by the perturbed runs
    assert rel[2][1] < 1e-5 * choices
    assert rel[2][2] < 1e-4, rel


# ----------------------------------------------------------- long runs
def _totals(d):
    m = d["m"].double()
    v = [d[k].double() for k in ("vx", "vy", "vz")]
    e = 0.5 * m * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2) + m * d["u"].double()
    return [float((m * vv).sum()) for vv in v], float(e.sum()), float((m * (v[0].abs() + v[1].abs() + v[2].abs())).sum())


def test_turbulence_400_fp32_steps_conserve_momentum_and_energy():
    """400 FP32 CFL steps of 64^3 turbulence (about t = 0.5, half a sound
    crossing): every pair's momentum and energy contributions are bitwise
    opposite and the rates are summed in FP64, so the totals drift only by
    the rounding of the FP32 state update (about 1e-9 here); the status
    word stays clean throughout."""
    m = gz()
    q = I.turbulence(64, seed=11)
    ctx = m.Context([q.N], m.default_params(precision=m.GZ_MIXED32))
    d = m.to_device(q, m.GZ_MIXED32)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    p0, e0, scale = _totals(d)
    t = 0.0
    for s in range(400):
        ctx.step(d, 0.0, dt)
        t += float(dt.item())
        if s % 100 == 99:
            st = ctx.status(reset=True)
            assert st["ok"], (s, st)
    p1, e1, _ = _totals(d)
    drift_p = max(abs(a - b) for a, b in zip(p1, p0)) / scale
    drift_e = abs(e1 - e0) / abs(e0)
    print(f"t = {t:.3f}: momentum drift {drift_p:.2e} of sum m|v|, energy drift {drift_e:.2e}")
    assert t > 0.3
    assert drift_p < 1e-7 and drift_e < 1e-7
    ctx.close()


def test_ensemble_200_steps_keep_a_clean_status():
    """The 256-box ensemble (Sod tubes and Sedov blasts, 8^3 to 24^3) over 200
    FP32 steps with the 48-entry density cache: no status bit (no
    non-convergence, list overflow or non-finite value) as the blasts empty
    their centres and particles leave the cache for the warp kernel."""
    m = gz()
    ens = I.ensemble(256, seed=1716)
    counts = [int(c) for c in ens.counts]
    ctx = m.Context(counts, m.default_params(precision=m.GZ_MIXED32, density_cache=48))
    d = m.to_device(ens, m.GZ_MIXED32)
    dt = torch.zeros(len(counts), dtype=torch.float64, device="cuda")
    for s in range(200):
        ctx.step(d, 0.0, dt)
        if s % 50 == 49:
            st = ctx.status(reset=True)
            assert st["ok"], (s, st)
    assert bool(torch.isfinite(d["u"]).all()) and bool((d["u"] > 0).all())
    ctx.close()
