"""Pins of the oracle's hierarchical (power-of-two) timesteps (reading HT):
K = 0 is the global step bitwise; an interval short enough for every
particle's criterion is one global step whatever K; momentum and energy are
conserved over an interval with mixed bins (pairwise exchange with
power-of-two shares); a pair's two shares are equal and opposite when its
particles sit in different bins; the Sedov blast keeps the global-step
accuracy with a fraction of the particle updates."""
import numpy as np
import pytest

import oracle as O
from paper_1712_01294_gb300 import inputs as I

from test_oracle_pins import state

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "u", "H")


def totals(s):
    P = np.array([(s.m * s.vx).sum(), (s.m * s.vy).sum(), (s.m * s.vz).sum()])
    E = (s.m * (s.u + 0.5 * (s.vx ** 2 + s.vy ** 2 + s.vz ** 2))).sum()
    return P, E


@pytest.mark.parametrize("kind", ["turb", "sedov"])
def test_k0_is_the_global_step_bitwise(kind):
    s = state(I.turbulence(11, seed=2) if kind == "turb" else I.sedov(11))
    a, dta, _, _, _ = O.step(s, O.params())
    b, D, bins, na = O.step_hier(s, O.params(), 0)
    assert D == dta and na == s.N and not bins.any()
    for k in FIELDS:
        assert np.array_equal(getattr(a, k), getattr(b, k)), k


def test_interval_within_every_criterion_is_one_global_step():
    s = state(I.turbulence(10, seed=4))
    p = O.params()
    _, dt_cfl, _, _, _ = O.step(s, p)
    D = 0.5 * dt_cfl  # every particle fits bin 0; substeps 1..7 are empty
    a, _, _, _, _ = O.step(s, p, dt=D)
    b, Db, bins, na = O.step_hier(s, p, 3, dt=D)
    assert Db == D and not bins.any() and na == s.N
    for k in FIELDS:
        assert np.array_equal(getattr(a, k), getattr(b, k)), k


@pytest.mark.parametrize("kind,K", [("turb", 2), ("sedov", 4)])
def test_interval_conserves_momentum_and_energy(kind, K):
    s = state(I.turbulence(10, seed=5) if kind == "turb" else I.sedov(12))
    P0, E0 = totals(s)
    c = O.Counters()
    o, D, bins, na = O.step_hier(s, O.params(), K, counters=c)
    assert len(np.unique(bins)) > 1  # mixed bins
    assert c.ufloor == 0
    P1, E1 = totals(o)
    scale = (s.m * np.sqrt(s.vx ** 2 + s.vy ** 2 + s.vz ** 2)).sum() + (s.m * np.sqrt(s.u)).sum()
    assert np.all(np.abs(P1 - P0) <= 1e-13 * scale), (P1 - P0)
    assert E1 == pytest.approx(E0, rel=1e-13)


def test_pair_shares_in_different_bins_are_equal_and_opposite():
    rng = np.random.default_rng(8)
    nonzero = 0
    for _ in range(20):
        x = np.array([0.5, 0.5 + rng.uniform(-0.05, 0.05)])
        y = np.array([0.5, 0.5 + rng.uniform(-0.05, 0.05)])
        z = np.array([0.5, 0.5 + rng.uniform(-0.05, 0.05)])
        ids = np.array([3, 9], dtype=np.int64)
        H = np.array([0.12, 0.1])
        n = np.array([900.0, 1100.0])
        m = np.array([1e-3, 2e-3])
        v = rng.normal(0, 0.2, (3, 2))
        u = rng.uniform(0.5, 2, 2)
        grad = rng.normal(0, 0.3, (15, 2))
        B = np.zeros((6, 2))
        B[0] = B[3] = B[5] = 300.0
        bins = np.array(rng.permutation([1, 3]), dtype=np.int32)
        active = np.array([1, 0], dtype=np.uint8) if bins[0] > bins[1] else np.array([0, 1], np.uint8)
        D = 0.01
        accp, accE, tch = O.exchange(x, y, z, ids, m, H, n, v[0], v[1], v[2], u, grad, B, bins, active, D)
        dt = D / 2.0 ** bins
        assert np.all(tch == 1)
        for r in range(3):
            assert accp[r, 0] * dt[0] == -accp[r, 1] * dt[1]
        assert accE[0] * dt[0] == -accE[1] * dt[1]
        nonzero += accE[0] != 0.0
    assert nonzero >= 15


@pytest.mark.slow
def test_sedov_blast_keeps_global_step_accuracy_with_fewer_updates():
    sedov_exact = pytest.importorskip("sedov_exact")
    res = {}
    for K in (0, 3):
        s = state(I.sedov(18))
        t, work = 0.0, 0
        while t < 0.04:
            s, D, _, na = O.step_hier(s, O.params(), K)
            t += D
            work += na
        H, nn, _, _ = O.density(s, O.params())
        rho = s.m * nn
        r = np.sqrt((s.x - 0.5) ** 2 + (s.y - 0.5) ** 2 + (s.z - 0.5) ** 2)
        keep = r < 0.5
        b = np.minimum((r[keep] / 0.5 * 50).astype(int), 49)
        prof = np.bincount(b, rho[keep], 50) / np.maximum(np.bincount(b, None, 50), 1)
        R = (np.argmax(prof) + 0.5) * 0.01
        res[K] = (R / sedov_exact.shock_radius(t), work / s.N)
    assert abs(res[0][0] - 1.0) < 0.1
    assert abs(res[3][0] - res[0][0]) < 0.03
    assert res[3][1] < 0.5 * res[0][1]


def test_mfv_k0_is_the_global_mfv_step_bitwise():
    s = state(I.turbulence(10, seed=9))
    p = O.params(scheme=O.MFV)
    a, dta, _, _, _ = O.step(s, p)
    b, D, bins, na = O.step_hier(s, p, 0)
    assert D == dta
    for k in FIELDS + ("m",):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k


def test_mfv_interval_conserves_mass_momentum_energy():
    s = state(I.sedov(12))
    P0, E0 = totals(s)
    M0 = s.m.sum()
    o, D, bins, na = O.step_hier(s, O.params(scheme=O.MFV), 3)
    assert len(np.unique(bins)) > 1
    assert np.abs(o.m - s.m).max() > 0.0  # mass moved
    assert o.m.sum() == pytest.approx(M0, rel=1e-14)
    P1, E1 = totals(o)
    scale = (s.m * np.sqrt(s.vx ** 2 + s.vy ** 2 + s.vz ** 2)).sum() + (s.m * np.sqrt(s.u)).sum()
    assert np.all(np.abs(P1 - P0) <= 1e-13 * scale)
    assert E1 == pytest.approx(E0, rel=1e-13)
