"""The benchmark's own launch at full size: one gz_step of the 128^3
turbulence box (2,097,152 particles, FP32 mixed path, one box, default cell
size), and of a 256^3 box, checked against the FP64 oracle on sampled
outputs it can compute one by one: every particle of four cubic sub-boxes (one of them around the
particle that sets the CFL step), each oracle pass run on the particles it
needs there (sub-box plus halos of 2.2 and 4.4 times the largest support).
Tolerances as in the per-pass parity tests.  FP32: H within 2e-6, per-particle
timesteps within 1e-5, the step's changes of v and u within 50 x 2e-5 of
their RMS (RMS error).  FP64 (the same launch in double): h-iteration counts
equal, H and timesteps within 1e-12, the changes within 1e-10 of their RMS
(max error)."""
import numpy as np
import pytest

import oracle as O
from paper_1712_01294_gb300 import inputs as I

from gpu_common import cast_state, device, field_err, min_image, ostate

pytestmark = pytest.mark.gpu


def around(s, centres, half):
    """Particles within `half` (per axis, periodic) of any centre."""
    ok = np.zeros(s.N, dtype=bool)
    for c in centres:
        m = np.ones(s.N, dtype=bool)
        for k, ck in zip(("x", "y", "z"), c):
            m &= np.abs(min_image(getattr(s, k) - ck)) < half
        ok |= m
    return ok


def sampled_step_check(n, prec):
    import torch

    import paper_1712_01294_gb300 as m
    f64 = prec == m.GZ_FP64
    q = cast_state(I.turbulence(n, seed=1714), prec)
    s = ostate(q)
    ctx = m.Context([q.N], m.default_params(precision=prec))
    # per-pass view of the step's first passes: converged H, n, per-particle dt
    dc = device(q, prec)
    n_g, it_g = ctx.density(dc)
    it_g = it_g.cpu().numpy()
    dti, dtb = ctx.timestep(dc, n_g)
    H_g = dc["h"].cpu().numpy().astype(np.float64)
    dti = dti.cpu().numpy()
    kmin = int(np.argmin(dti))
    # the step itself, as the benchmark launches it
    d = device(q, prec)
    dtu = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.step(d, 0.0, dtu)
    st = ctx.status(reset=True)
    assert st["ok"], st
    dt = float(dtu.item())
    assert dt == float(dtb[0].item())

    rng = np.random.default_rng(n)
    centres = [rng.uniform(0, 1, 3) for _ in range(3)] + [np.array([s.x[kmin], s.y[kmin], s.z[kmin]])]
    half = 0.02
    Hm = 1.3 * float(np.max(s.H))
    m_f, m_g, m_d = around(s, centres, half), around(s, centres, half + 2.2 * Hm), \
        around(s, centres, half + 4.4 * Hm)
    assert m_f.sum() > 300 and m_f[kmin]
    p = O.params()
    H, n, it_o, _ = O.density(s, p, mask=m_d)
    H = np.where(m_d, H, s.H)
    n = np.where(m_d, n, 1.0)
    assert np.max(np.abs(H_g[m_f] - H[m_f]) / H[m_f]) <= (1e-12 if f64 else 2e-6)
    if f64:
        assert np.array_equal(it_g[m_f], it_o[m_f])
    g = O.gradients(s, H, n, p, mask=m_g)
    dti_o, _ = O.timestep(s, H, n, p, mask=m_f)
    tol_dt = 1e-12 if f64 else 1e-5
    assert np.max(np.abs(dti[m_f] - dti_o[m_f]) / dti_o[m_f]) <= tol_dt
    assert abs(dt - p.cfl * dti_o[kmin]) <= tol_dt * dt  # the box's CFL step
    dp, dE = O.fluxes(s, H, n, g["grad"], g["B"], dt, p, mask=m_f)
    o = O.update(s, dp, dE, dt, p)
    for k in ("vx", "vy", "vz", "u"):
        got = d[k].cpu().numpy().astype(np.float64)[m_f] - getattr(s, k)[m_f]
        ref = getattr(o, k)[m_f] - getattr(s, k)[m_f]
        mx, rm = field_err(got, ref)
        assert (mx <= 1e-10) if f64 else (rm <= 50 * 2e-5), (k, mx, rm)
    for k in ("x", "y", "z"):
        got = min_image(d[k].cpu().numpy().astype(np.float64)[m_f] - getattr(s, k)[m_f])
        ref = min_image(getattr(o, k)[m_f] - getattr(s, k)[m_f])
        mx, rm = field_err(got, ref)
        assert (mx <= 1e-10) if f64 else (rm <= 50 * 2e-5), (k, mx, rm)
    assert np.max(np.abs(d["h"].cpu().numpy().astype(np.float64)[m_f] - H[m_f]) / H[m_f]) <= \
        (1e-12 if f64 else 2e-6)
    ctx.close()


@pytest.mark.parametrize("prec", [1, 0])
def test_128cubed_step_matches_oracle_on_sampled_sub_boxes(prec):
    sampled_step_check(128, prec)


def test_256cubed_fp32_step_matches_oracle_on_sampled_sub_boxes():
    """The same check at 256^3 = 16,777,216 particles (about 18 GB of
    context on the device): indices, list layouts and the 24-bit sort keys
    at eight times the benchmark's size."""
    import paper_1712_01294_gb300 as m
    sampled_step_check(256, m.GZ_MIXED32)


@pytest.mark.parametrize("prec", [0, 1])
def test_128cubed_adjoint_of_conserved_totals(prec):
    """Total momentum and total energy after a step do not depend on the
    positions and equal their values before it, whatever the state (pairwise
    equal and opposite fluxes), so the adjoint of the step, seeded with their
    derivatives (m and m v; m), must return m for the velocities, m v and m
    for velocities and u, and zero for the positions.  A property of the full
    launch that holds at any size; checked at the benchmark's 128^3."""
    import torch

    import paper_1712_01294_gb300 as m
    q = cast_state(I.turbulence(128, seed=1714), prec)
    ctx = m.Context([q.N], m.default_params(precision=prec))
    T = torch.float64 if prec == 0 else torch.float32
    start = device(q, prec)
    fwd = device(q, prec)
    lvl = m.GZ_CKPT_GRADIENTS
    ck = ctx.new_checkpoint(lvl)
    dtu = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.step(fwd, 0.0, dtu, ck, lvl)
    dt = float(dtu.item())
    start["h"] = fwd["h"]
    mass = start["m"]
    zeros = lambda: torch.zeros(q.N, dtype=T, device="cuda")
    tol = 1e-10 if prec == 0 else 2e-4
    rms = lambda a: float(a.double().pow(2).mean().sqrt())
    # scale of the position and energy adjoints: a functional with no
    # conservation law, L = sum r_i vx_i' with random weights r
    gend = {k: zeros() for k in ("x", "y", "z", "vx", "vy", "vz", "u")}
    gend["vx"] = (mass * torch.randn(q.N, generator=torch.Generator(device="cuda").manual_seed(3),
                                     device="cuda", dtype=torch.float64).to(T))
    ref = {k: zeros() for k in ("x", "y", "z", "vx", "vy", "vz", "u", "m")}
    ctx.step_backward(start, dt, gend, ref, ck, lvl)
    assert rms(ref["x"]) > 0 and rms(ref["u"]) > 0
    # momentum (x component): L = sum m vx'
    gend = {k: zeros() for k in ("x", "y", "z", "vx", "vy", "vz", "u")}
    gend["vx"] = mass.clone()
    gs = {k: zeros() for k in ("x", "y", "z", "vx", "vy", "vz", "u", "m")}
    ctx.step_backward(start, dt, gend, gs, ck, lvl)
    assert ctx.status(reset=True)["ok"]
    rel = lambda a, b: float((a.double() - b.double()).norm() / b.double().norm())
    assert rel(gs["vx"], mass) <= tol
    for k in ("x", "y", "z", "vy", "vz", "u"):
        assert rms(gs[k]) <= tol * rms(ref[k] if k in ("x", "y", "z", "u") else ref["vx"]), k
    # total energy: L = sum m (u' + |v'|^2 / 2)
    gend = {k: zeros() for k in ("x", "y", "z")}
    for k in ("vx", "vy", "vz"):
        gend[k] = mass * fwd[k]
    gend["u"] = mass.clone()
    gs = {k: zeros() for k in ("x", "y", "z", "vx", "vy", "vz", "u", "m")}
    ctx.step_backward(start, dt, gend, gs, ck, lvl)
    assert ctx.status(reset=True)["ok"]
    for k in ("vx", "vy", "vz"):
        assert rel(gs[k], mass * start[k]) <= 10 * tol, k
    assert rel(gs["u"], mass) <= tol
    for k in ("x", "y", "z"):
        assert rms(gs[k]) <= 10 * tol * rms(ref[k]) * rms(fwd["vx"]), k  # seeds m v against m r
