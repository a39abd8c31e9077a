"""Pins of the oracle's MFV variant (faces moving with the interpolated frame
velocity v_f, HLLC mass, momentum and energy fluxes, evolving masses) against
what the mathematics fixes: the physical Euler flux for equal states, the
exact Godunov flux for weak jumps (HLLC's error is second order in the jump),
Galilean covariance of the flux through a moving face, pairwise conservation
of mass, momentum and energy, a uniform flow staying uniform, and Sod."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1712_01294_gb300 import inputs as I

from test_oracle_pins import sod_exact_rho, state

GAM = 5.0 / 3.0


def euler_flux(W, vf, n, g=GAM):
    """Lab-frame flux densities through a face moving with vf, normal n."""
    rho, v, P = W[0], np.asarray(W[1:4]), W[4]
    un = (v - vf) @ n
    E = P / (g - 1.0) + 0.5 * rho * (v @ v)
    return rho * un, rho * v * un + P * n, E * un + P * (v @ n)


def test_equal_states_give_the_physical_flux():
    rng = np.random.default_rng(3)
    for _ in range(20):
        W = np.array([rng.uniform(0.5, 2), *rng.normal(0, 1, 3), rng.uniform(0.5, 2)])
        vf = rng.normal(0, 0.5, 3)
        n = rng.normal(0, 1, 3)
        n /= np.linalg.norm(n)
        Fm, Fp, FE = O.hllc_flux(W, W, vf, n, GAM)
        em, ep, eE = euler_flux(W, vf, n)
        assert Fm == pytest.approx(em, rel=1e-12, abs=1e-14)
        assert np.allclose(Fp, ep, rtol=1e-12, atol=1e-14)
        assert FE == pytest.approx(eE, rel=1e-12, abs=1e-14)


def exact_godunov(rL, uL, PL, rR, uR, PR, g=GAM):
    r, u, P = O.riemann_sample(rL, uL, PL, rR, uR, PR, g, 0.0)[:, 0]
    E = P / (g - 1.0) + 0.5 * r * u * u
    return np.array([r * u, r * u * u + P, u * (E + P)])


def test_weak_jumps_converge_to_the_exact_godunov_flux_at_second_order():
    errs = []
    for eps in (1e-2, 1e-3):
        L = (1.0, 0.3, 1.0)
        R = (1.0 + eps, 0.3 - 0.5 * eps, 1.0 + 2 * eps)
        Fm, Fp, FE = O.hllc_flux([L[0], L[1], 0, 0, L[2]], [R[0], R[1], 0, 0, R[2]],
                                 [0, 0, 0], [1, 0, 0], GAM)
        h = np.array([Fm, Fp[0], FE])
        e = exact_godunov(*L, *R)
        errs.append(float(np.max(np.abs(h - e) / np.abs(e))))
    assert errs[0] < 1e-4
    assert errs[1] < 0.02 * errs[0]  # a tenth of the jump, a hundredth of the error


def test_flux_is_galilean_covariant():
    rng = np.random.default_rng(5)
    WL = np.array([1.2, 0.3, -0.2, 0.1, 1.4])
    WR = np.array([0.7, -0.1, 0.4, 0.2, 0.6])
    vf = np.array([0.1, 0.05, -0.02])
    n = np.array([0.48, 0.6, 0.64])
    n /= np.linalg.norm(n)
    Fm, Fp, FE = O.hllc_flux(WL, WR, vf, n, GAM)
    for _ in range(5):
        v0 = rng.normal(0, 1, 3)
        b = lambda W: np.array([W[0], *(W[1:4] + v0), W[4]])
        Gm, Gp, GE = O.hllc_flux(b(WL), b(WR), vf + v0, n, GAM)
        assert Gm == pytest.approx(Fm, rel=1e-12, abs=1e-14)
        assert np.allclose(Gp, Fp + v0 * Fm, rtol=1e-12, atol=1e-13)
        assert GE == pytest.approx(FE + v0 @ Fp + 0.5 * (v0 @ v0) * Fm, rel=1e-11, abs=1e-13)


def test_rates_and_step_conserve_mass_momentum_energy():
    s = state(I.turbulence(10, seed=7))
    p = O.params(scheme=O.MFV)
    H, n, _, _ = O.density(s, p)
    g = O.gradients(s, H, n, p)
    _, dt = O.timestep(s, H, n, p)
    dp, dE, dm = O.fluxes(s, H, n, g["grad"], g["B"], dt, p, with_mass=True)
    assert abs(dm.sum()) <= 1e-13 * np.abs(dm).sum()
    assert np.all(np.abs(dp.sum(1)) <= 1e-13 * np.abs(dp).sum(1))
    assert abs(dE.sum()) <= 1e-13 * np.abs(dE).sum()
    assert np.abs(dm).sum() > 0.0  # MFV moves mass between particles
    M0 = s.m.sum()
    P0 = np.array([(s.m * s.vx).sum(), (s.m * s.vy).sum(), (s.m * s.vz).sum()])
    E0 = (s.m * (s.u + 0.5 * (s.vx ** 2 + s.vy ** 2 + s.vz ** 2))).sum()
    o, dt2, _, _, _, dm2 = O.step(s, p, with_mass=True)
    assert np.abs(dm2).sum() > 0.0
    assert o.m.sum() == pytest.approx(M0, rel=1e-14)
    P1 = np.array([(o.m * o.vx).sum(), (o.m * o.vy).sum(), (o.m * o.vz).sum()])
    E1 = (o.m * (o.u + 0.5 * (o.vx ** 2 + o.vy ** 2 + o.vz ** 2))).sum()
    assert np.all(np.abs(P1 - P0) <= 1e-13 * (np.abs(s.m * s.vx).sum() + 1.0))
    assert E1 == pytest.approx(E0, rel=1e-13)


def test_uniform_flow_on_a_perfect_lattice_has_zero_rates():
    n = 8
    x, y, z, _ = I.lattice(n, np.random.default_rng(0), 0.0)
    N = x.size
    v0 = np.array([0.3, -0.2, 0.1])
    s = O.State(x, y, z, np.full(N, v0[0]), np.full(N, v0[1]), np.full(N, v0[2]),
                np.full(N, 1.0 / N), np.full(N, 1.5), np.full(N, I.h0(N)), np.arange(N))
    p = O.params(scheme=O.MFV)
    H, nn, _, _ = O.density(s, p)
    g = O.gradients(s, H, nn, p)
    dp, dE, dm = O.fluxes(s, H, nn, g["grad"], g["B"], 1e-3, p, with_mass=True)
    assert np.max(np.abs(dm)) <= 1e-12
    assert np.max(np.abs(dp)) <= 1e-12
    assert np.max(np.abs(dE)) <= 1e-12


def sod_l1_mfv(n, t_end=0.1):
    s = state(I.sod(n))
    p = O.params(scheme=O.MFV)
    t = 0.0
    while t < t_end - 1e-12:
        H, nn, _, _ = O.density(s, p)
        _, dt = O.timestep(s, H, nn, p)
        dt = min(dt, t_end - t)
        s, dt, _, _, _ = O.step(s, p, dt=dt)
        t += dt
    H, nn, _, _ = O.density(s, p)
    rho = s.m * nn
    bins = np.floor(s.x * n).astype(int)
    rb = np.bincount(bins, rho, n) / np.bincount(bins, None, n)
    xf = (np.arange(n)[:, None] + (np.arange(16) + 0.5)[None, :] / 16) / n
    ex = sod_exact_rho(xf.ravel(), t).reshape(n, 16).mean(1)
    return float(np.mean(np.abs(rb - ex)))


@pytest.mark.slow
def test_mfv_sod_approaches_the_exact_solution():
    e16 = sod_l1_mfv(16)
    e32 = sod_l1_mfv(32)
    assert e16 < 0.08
    assert e32 < 0.06 and e32 < e16
