"""Sedov-Taylor point blast (strong explosion in a uniform cold gas), the
self-similar solution written out from the Euler equations: test reference
for the shock radius R(t) = xi0 (E t^2 / rho0)^(1/5).

With R(t), D = dR/dt = 2R / (5t), eta = r / R and u = D U(eta),
rho = rho0 G(eta), P = rho0 D^2 Pi(eta), the spherical Euler equations become
    (U - eta) G' + G U'            = -2 G U / eta          (mass)
    (U - eta) U' + Pi' / G         = (3/2) U               (momentum)
    (U - eta) (Pi'/Pi - gamma G'/G) = 3                    (entropy)
with the strong-shock jump conditions at eta = 1: U = Pi = 2/(gamma+1),
G = (gamma+1)/(gamma-1).  Energy conservation, E = 4 pi rho0 D^2 R^3 I with
I = int_0^1 (G U^2 / 2 + Pi / (gamma-1)) eta^2 d eta and D^2 R^3 =
(4/25) R^5 / t^2, gives xi0 = (25 / (16 pi I))^(1/5).
"""
import numpy as np
from scipy.integrate import solve_ivp


def _rhs(gam):
    def f(eta, y):
        U, G, P, _ = y
        a = U - eta
        Up = (1.5 * U - (P / (G * a)) * (3.0 - 2.0 * gam * U / eta)) / (a - gam * P / (G * a))
        Gp = (-2.0 * G * U / eta - G * Up) / a
        Pp = P * (3.0 / a + gam * Gp / G)
        return [Up, Gp, Pp, -(0.5 * G * U * U + P / (gam - 1.0)) * eta * eta]
    return f


def profile(gam, eta_min=1e-3):
    """Integrates from the shock inwards; returns (eta, U, G, Pi, I)."""
    y0 = [2.0 / (gam + 1.0), (gam + 1.0) / (gam - 1.0), 2.0 / (gam + 1.0), 0.0]
    sol = solve_ivp(_rhs(gam), (1.0, eta_min), y0, rtol=1e-11, atol=1e-14, method="LSODA",
                    dense_output=False)
    if sol.status != 0:
        raise RuntimeError(sol.message)
    return sol.t, sol.y[0], sol.y[1], sol.y[2], sol.y[3, -1]


def xi0(gam):
    return (25.0 / (16.0 * np.pi * profile(gam)[4])) ** 0.2


def shock_radius(t, E=1.0, rho0=1.0, gam=5.0 / 3.0):
    return xi0(gam) * (E * t * t / rho0) ** 0.2
