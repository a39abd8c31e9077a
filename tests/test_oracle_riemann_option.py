"""Pins of the oracle's Riemann-solver option for the MFM face (riemann =
EXACT on every face, EXACT_FALLBACK where HLLC's P* < 0) against closed forms:
the symmetric expansion (two rarefactions: u* = 0 and
P* = P (1 - (gamma-1) w / (2c))^(2 gamma/(gamma-1))), the symmetric collision
(two shocks: u* = 0 and (P* - P) sqrt(A/(P* + B)) = w, a quadratic), weak
jumps (the exact and HLLC stars agree to second order), and whole-step
properties (conservation; the fallback is HLLC itself where no P* < 0)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1712_01294_gb300 import inputs as I

from test_oracle_pins import state

G = 5.0 / 3.0


def face(WL, WR):
    """One face along +x between two particles with zero gradients, equal H
    and n, and B = identity: face states are the particle states."""
    base = {"H": 0.1, "n": 1000.0, "g": np.zeros(15), "B": np.array([1.0, 0, 0, 1.0, 0, 1.0])}
    L = dict(base, x=np.array([0.5, 0.5, 0.5]), W=np.asarray(WL, float))
    R = dict(base, x=np.array([0.55, 0.5, 0.5]), W=np.asarray(WR, float))
    return L, R


def run(L, R, riemann):
    return O.pair(L, R, 1e-3, O.params(hancock=0, riemann=riemann))


@pytest.mark.parametrize("w", [0.9, 1.5, 2.5])
def test_symmetric_expansion_matches_the_rarefaction_closed_form(w):
    rho, P = 1.0, 1.0
    c = math.sqrt(G * P / rho)
    exact = P * (1.0 - 0.5 * (G - 1.0) * w / c) ** (2.0 * G / (G - 1.0))
    L, R = face([rho, -w, 0, 0, P], [rho, w, 0, 0, P])
    h = run(L, R, O.HLLC)
    assert w <= c / G or h["pstar"] == 0.0  # HLLC-Davis: P - rho c w, clamped
    for mode in (O.EXACT, O.EXACT_FALLBACK):
        r = run(L, R, mode)
        assert r["pstar"] == pytest.approx(exact, rel=1e-12)
        assert abs(r["sstar"]) <= 1e-13
        # HLLC's P* < 0 is still reported under the fallback; never under EXACT
        assert bool(r["flags"] & 2) == (mode == O.EXACT_FALLBACK and w > c / G)
        # the MFM momentum rate is -P* A
        assert np.allclose(r["dp"], -r["pstar"] * r["A"], rtol=1e-14, atol=0)


@pytest.mark.parametrize("w", [0.3, 1.0, 3.0])
def test_symmetric_collision_matches_the_two_shock_closed_form(w):
    rho, P = 1.3, 0.7
    A = 2.0 / ((G + 1.0) * rho)
    B = (G - 1.0) / (G + 1.0) * P
    # (p - P)^2 A = w^2 (p + B), larger root
    a, b, cc = A, -(2.0 * A * P + w * w), A * P * P - w * w * B
    exact = (-b + math.sqrt(b * b - 4.0 * a * cc)) / (2.0 * a)
    L, R = face([rho, w, 0, 0, P], [rho, -w, 0, 0, P])
    r = run(L, R, O.EXACT)
    assert r["pstar"] == pytest.approx(exact, rel=1e-12)
    assert abs(r["sstar"]) <= 1e-13
    assert r["flags"] == 0
    # the fallback keeps HLLC where its P* is positive
    assert run(L, R, O.EXACT_FALLBACK)["pstar"] == run(L, R, O.HLLC)["pstar"]


def test_weak_jumps_exact_and_hllc_agree_to_second_order():
    errs = []
    for eps in (1e-2, 1e-3):
        L, R = face([1.0, 0.1, 0, 0, 1.0], [1.0 + eps, 0.1 - eps, 0.2, 0, 1.0 + 3 * eps])
        e = run(L, R, O.EXACT)
        h = run(L, R, O.HLLC)
        errs.append(max(abs(e["pstar"] - h["pstar"]), abs(e["sstar"] - h["sstar"])))
    assert errs[0] < 1e-4
    assert errs[1] < 0.02 * errs[0]


def test_vacuum_face_carries_no_pressure():
    # u_R - u_L = 6 > 2 (c_L + c_R)/(gamma - 1) = 4.9: the fans leave a vacuum
    L, R = face([1.0, -3.0, 0, 0, 0.4], [1.0, 3.0, 0, 0, 0.4])
    r = run(L, R, O.EXACT)
    assert r["pstar"] == 0.0 and r["flags"] & 2
    assert np.all(r["dp"] == 0.0) and r["dE"] == 0.0


def test_exact_fluxes_conserve_momentum_and_energy():
    s = state(I.turbulence(10, seed=3))
    p = O.params(riemann=O.EXACT)
    H, n, _, _ = O.density(s, p)
    g = O.gradients(s, H, n, p)
    _, dt = O.timestep(s, H, n, p)
    dp, dE = O.fluxes(s, H, n, g["grad"], g["B"], dt, p)
    assert np.all(np.abs(dp.sum(1)) <= 1e-13 * np.abs(dp).sum(1))
    assert abs(dE.sum()) <= 1e-13 * np.abs(dE).sum()
    dph, _ = O.fluxes(s, H, n, g["grad"], g["B"], dt, O.params())
    # a different solver of the same problems: Mach 0.5 jumps are not weak, so
    # the particle rates differ by ~10 % RMS, strongly correlated
    rms = lambda a: np.sqrt(np.mean(a * a))
    assert 0.0 < rms(dp - dph) <= 0.2 * rms(dph)
    assert np.corrcoef(dp.ravel(), dph.ravel())[0, 1] > 0.99


def test_fallback_is_hllc_without_negative_star_pressure_and_repairs_it_where_there_is():
    s = state(I.sod(12))
    a = O.step(s, O.params())[0]
    b = O.step(s, O.params(riemann=O.EXACT_FALLBACK))[0]
    for k in ("x", "vx", "u", "H"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
    s = state(I.sod(12, rho_l=1.0, p_l=0.4, rho_r=1.0, p_r=0.4, u_l=-2.0, u_r=2.0))
    c_h, c_f = O.Counters(), O.Counters()
    H, n, _, _ = O.density(s, O.params())
    g = O.gradients(s, H, n, O.params())
    _, dt = O.timestep(s, H, n, O.params())
    dp_h, _ = O.fluxes(s, H, n, g["grad"], g["B"], dt, O.params(), counters=c_h)
    dp_f, _ = O.fluxes(s, H, n, g["grad"], g["B"], dt, O.params(riemann=O.EXACT_FALLBACK),
                       counters=c_f)
    assert c_h.pstar_neg > 0 and c_f.pstar_neg == c_h.pstar_neg
    # the repaired faces carry the (small, positive) exact star pressure: the
    # rarefaction's pull on the particles grows
    assert not np.array_equal(dp_h, dp_f)


def test_mfv_refuses_the_exact_option():
    with pytest.raises(ValueError):
        O.params(scheme=O.MFV, riemann=O.EXACT)
