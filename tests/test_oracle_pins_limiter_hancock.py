"""Pins of two oracle readings that admissibility alone does not fix (no GPU).

O9, the per-particle limiter: alpha_f is the LARGEST factor in [0, 1] that
keeps every limited face value f_i + alpha g . (s_ij d_ij), j in N_i, inside
[f_i + beta (f_min - f_i), f_i + beta (f_max - f_i)] (extremes over N_i and i).
Where alpha_f < 1 some face value therefore sits on that bound: an admissible
but smaller factor (alpha / 2, a minimum over a wider set of pairs) leaves
every face strictly inside and fails here.

O11, the Hancock half step: the increment added to each side's face state is
the first-order Taylor term, over dt/2, of the exact Lagrangian evolution of
the Euler equations (D rho/Dt = -rho div v, D v/Dt = -grad P / rho,
D P/Dt = -gamma P div v).  Two flows whose Lagrangian evolution is known in
closed form pin it: a homologous flow v = D x at uniform rho, P (parcel
density rho0 / det(I + t D), pressure P0 det(I + t D)^-gamma, velocity
constant) and a gas at rest in a uniform pressure gradient c (parcel velocity
-c t / rho0, density and pressure constant).  The increments are read as the
oracle's face states at dt minus those at dt = 0 (same reconstruction), and
must match the closed forms at t = dt/2 with an error of order dt^2 (halving
dt quarters it).  A wrong sign, a step of dt instead of dt/2, a missing rho
or gamma factor, or a divergence formed from the wrong gradient components
fails.

The whole step's time order is recorded too: with the face geometry taken at
the start of the step and the pairwise clamp of O11 applied after the half
step, the step is first order in time (the clamp removes the increment on
faces whose two particles hold equal values); on a smooth monotone flow on a
perfect lattice the Hancock step's temporal error is nevertheless a quarter
of the first-order (hancock = 0) step's.
"""
import math

import numpy as np

import oracle as O
from paper_1712_01294_gb300 import inputs as I

GAM = 5.0 / 3.0


def _state(p):
    return O.State.from_any(p.__dict__)


# ------------------------------------------------------------- O9 limiter
def _limited_faces(s, beta):
    p = O.params(beta=beta)
    H, nn, _, _ = O.density(s, p)
    out = O.gradients(s, H, nn, p)
    off, nb = O.neighbours(s, H)
    W = np.stack([s.m * nn, s.vx, s.vy, s.vz, (GAM - 1) * s.m * nn * s.u])
    X = np.stack([s.x, s.y, s.z], 1)
    return H, out, off, nb, W, X


def _check_alpha_is_maximal(s, beta):
    H, out, off, nb, W, X = _limited_faces(s, beta)
    # the limited gradient is alpha times the raw one
    assert np.array_equal(out["grad"], np.repeat(out["alpha"], 3, axis=0) * out["grad_raw"])
    touched = limited = 0
    for i in range(s.N):
        js = nb[off[i]:off[i + 1]]
        if js.size == 0:
            continue
        d = X[js] - X[i]
        d = np.where(d >= 0.5, d - 1.0, np.where(d < -0.5, d + 1.0, d))
        sd = d * (H[i] / (H[i] + H[js]))[:, None]
        for q in range(5):
            f = W[q]
            up = beta * (max(f[i], f[js].max()) - f[i])    # >= 0
            dn = beta * (min(f[i], f[js].min()) - f[i])    # <= 0
            inc = sd @ out["grad"][q * 3:q * 3 + 3, i]       # limited face value - f_i
            tol = 1e-11 * (up - dn) + 1e-14 * abs(f[i]) + 1e-300
            # admissible: every face inside the bounds
            assert np.all(inc <= up + tol) and np.all(inc >= dn - tol), (i, q)
            if out["alpha"][q, i] < 1.0:
                limited += 1
                # maximal: a face sits on a bound
                on_bound = (abs(inc.max() - up) <= tol) or (abs(inc.min() - dn) <= tol)
                assert on_bound, (i, q, out["alpha"][q, i], inc.max() - up, inc.min() - dn)
                touched += 1
    assert limited > 50 and touched == limited


def test_limiter_alpha_is_the_largest_admissible_factor_sedov():
    _check_alpha_is_maximal(_state(I.sedov(10)), 1.0)


def test_limiter_alpha_is_the_largest_admissible_factor_turbulence():
    _check_alpha_is_maximal(_state(I.turbulence(10, seed=41)), 1.0)


def test_limiter_beta_scales_the_admissible_band():
    # beta = 1/2: the band is half the neighbour range; limited faces reach
    # exactly half way to the extreme
    _check_alpha_is_maximal(_state(I.sedov(10)), 0.5)


def test_limiter_alpha_is_one_where_no_face_reaches_a_bound():
    # the reverse implication: alpha = 1 exactly when the raw faces stay inside
    s = _state(I.turbulence(10, seed=43))
    H, out, off, nb, W, X = _limited_faces(s, 1.0)
    for i in range(0, s.N, 7):
        js = nb[off[i]:off[i + 1]]
        d = X[js] - X[i]
        d = np.where(d >= 0.5, d - 1.0, np.where(d < -0.5, d + 1.0, d))
        sd = d * (H[i] / (H[i] + H[js]))[:, None]
        for q in range(5):
            f = W[q]
            up = max(f[i], f[js].max()) - f[i]
            dn = min(f[i], f[js].min()) - f[i]
            raw = sd @ out["grad_raw"][q * 3:q * 3 + 3, i]
            inside = np.all(raw < up) and np.all(raw > dn)
            outside = np.any(raw > up * (1 + 1e-9) + 1e-300) or np.any(raw < dn * (1 + 1e-9) - 1e-300)
            if inside:
                assert out["alpha"][q, i] == 1.0
            if outside:
                assert out["alpha"][q, i] < 1.0


# --------------------------------------------------------- O11 Hancock
def _side(x, W, g, H=0.1, n=1000.0):
    return dict(x=np.asarray(x, float), H=H, n=n, W=np.asarray(W, float),
                g=np.asarray(g, float), B=np.array([1.0, 0.0, 0.0, 1.0, 0.0, 1.0]) * 3e3)


def _increments(L, R, dt):
    """Hancock increments of both sides: face states at dt minus at dt = 0."""
    p = O.params(hancock=1)
    a = O.pair(L, R, dt, p)
    b = O.pair(L, R, 0.0, p)
    assert a["ok"] and b["ok"]
    return a["pred_L"] - b["pred_L"], a["pred_R"] - b["pred_R"]


def _homologous_pair(rho0, P0, D, v0):
    # rho, P uniform; v = v0 + D x: gradient rows d v_a / d x_b = D[a, b]
    g = np.zeros(15)
    g[3:12] = np.asarray(D, float).ravel()
    xL = np.array([0.41, 0.52, 0.47])
    xR = xL + np.array([0.031, -0.012, 0.022])
    WL = np.concatenate([[rho0], v0 + D @ xL, [P0]])
    WR = np.concatenate([[rho0], v0 + D @ xR, [P0]])
    return _side(xL, WL, g, H=0.052), _side(xR, WR, g, H=0.047)


def test_hancock_half_step_matches_homologous_flow():
    rho0, P0 = 2.5, 0.7
    D = np.array([[0.8, 0.3, -0.2], [-0.4, -0.35, 0.5], [0.25, 0.1, 0.6]])  # trace 1.05
    L, R = _homologous_pair(rho0, P0, D, np.array([0.1, -0.2, 0.05]))
    errs = []
    for dt in (0.02, 0.01, 0.005):
        t = 0.5 * dt
        J = np.linalg.det(np.eye(3) + t * D)
        exact = np.array([rho0 / J - rho0, 0.0, 0.0, 0.0, P0 * J ** (-GAM) - P0])
        iL, iR = _increments(L, R, dt)
        for inc in (iL, iR):
            # right sign and leading magnitude (compression/expansion of the parcel)
            assert np.sign(inc[0]) == np.sign(exact[0]) and np.sign(inc[4]) == np.sign(exact[4])
            assert np.all(np.abs(inc[1:4]) <= 1e-15)          # no pressure gradient: no kick
        errs.append(np.abs(np.concatenate([iL - exact, iR - exact])).max())
        # the error is second order: well below the increment itself
        assert errs[-1] <= 0.5 * (t * 1.05) ** 2 * max(rho0, GAM * (GAM + 1) * P0) * 4
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_hancock_half_step_matches_uniform_pressure_gradient():
    rho0, P0 = 2.5, 1.3
    c = np.array([0.3, -0.2, 0.5])
    g = np.zeros(15)
    g[12:15] = c
    xL = np.array([0.41, 0.52, 0.47])
    xR = xL + np.array([-0.02, 0.025, 0.03])
    L = _side(xL, [rho0, 0, 0, 0, P0 + c @ xL], g, H=0.05)
    R = _side(xR, [rho0, 0, 0, 0, P0 + c @ xR], g, H=0.055)
    for dt in (0.02, 0.004):
        iL, iR = _increments(L, R, dt)
        exact = np.concatenate([[0.0], -c * (0.5 * dt) / rho0, [0.0]])  # exact at any dt
        for inc in (iL, iR):
            assert np.allclose(inc, exact, rtol=1e-13, atol=1e-16), (inc, exact)


def test_hancock_off_adds_nothing_and_clamp_bounds_the_faces():
    rho0, P0 = 1.4, 0.9
    D = np.array([[0.5, 0.1, 0.0], [0.0, -0.3, 0.2], [0.1, 0.0, 0.4]])
    L, R = _homologous_pair(rho0, P0, D, np.zeros(3))
    L["W"][0], R["W"][0] = 1.3, 1.6        # unequal densities: a non-degenerate band
    off = O.pair(L, R, 0.05, O.params(hancock=0))
    zero = O.pair(L, R, 0.0, O.params(hancock=0))
    assert np.array_equal(off["pred_L"], zero["pred_L"]) and np.array_equal(off["pred_R"], zero["pred_R"])
    on = O.pair(L, R, 0.05, O.params(hancock=1))
    lo, hi = np.minimum(L["W"], R["W"]), np.maximum(L["W"], R["W"])
    for k in ("face_L", "face_R"):
        assert np.all(on[k] >= lo) and np.all(on[k] <= hi)
    # where the band is degenerate (equal pressures) the clamp removes the increment
    assert on["face_L"][4] == P0 and on["pred_L"][4] != P0


def _monotone_flow(n, a):
    s = _state(I.sod(n, jitter=0.0, rho_l=1.0, rho_r=1.0, p_l=1.0, p_r=1.0))
    X = np.sin(math.pi * (s.x - 0.5))
    Y = np.sin(math.pi * (s.y - 0.5))
    rho = 1.5 + a * X + 0.5 * a * Y
    P = 1.0 - a * X + 0.3 * a * Y
    s.vx = 0.8 * a * X + 0.2 * a * Y
    s.vy = -0.5 * a * X + 0.4 * a * Y
    s.vz = 0.3 * a * X
    s.m = s.m * rho
    s.u = P / ((GAM - 1) * rho)
    return s


def test_hancock_reduces_the_temporal_error_of_the_step():
    # successive differences of runs to the same time with m and 2m steps
    # measure the temporal error; the interior (monotone fields, away from the
    # fields' turning points at the box edge and the waves they send) is compared
    n, a, T = 24, 0.05, 0.02
    s = _monotone_flow(n, a)
    H, _, _, _ = O.density(s, O.params())
    s.H = H
    margin = 3 * H.max() + 2.4 * T
    inner = (np.abs(s.x - 0.5) < 0.5 - margin) & (np.abs(s.y - 0.5) < 0.5 - margin)
    assert inner.sum() > 1000

    def run(p, m):
        cur = s
        for _ in range(m):
            cur = O.step(cur, p, dt=T / m)[0]
        return cur

    def diff(u, v):
        return np.sqrt(np.mean(((u.vx - v.vx) ** 2 + (u.vy - v.vy) ** 2 + (u.u - v.u) ** 2)[inner]))

    e = {}
    for hk in (1, 0):
        p = O.params(hancock=hk)
        r4, r8, r16 = run(p, 4), run(p, 8), run(p, 16)
        e[hk] = (diff(r4, r8), diff(r8, r16))
    # first order without the half step (halving dt halves the difference)
    assert 1.8 < e[0][0] / e[0][1] < 2.2
    # with it the temporal error is a quarter of that (at most 0.35)
    assert e[1][1] < 0.35 * e[0][1] and e[1][0] < 0.45 * e[0][0]
