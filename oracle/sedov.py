"""Self-similar solution of a strong point explosion in a uniform ideal gas
at rest (the Sedov-Taylor blast wave).

TEST INFRASTRUCTURE ONLY: the analytic reference for the Sedov-blast setup
of Section 4.2.  Only ``tests/`` may use it; it shares no code with the
CUDA library.

Derivation (spherical Euler equations, energy E released at r = 0 into a
gas of density rho0 and negligible pressure): the shock radius is
R(t) = xi0 (E t^2 / rho0)^(1/5) and, with eta = r/R,
    u = R' U(eta),   rho = rho0 G(eta),   p = rho0 R'^2 P(eta).
Continuity, momentum and the entropy of each fluid element (p rho^-gamma
constant along it) become, with a = R'/R = 2/(5t),
    (U - eta) U' + P'/G = 3 U / 2
    G U' + (U - eta) G' = -2 G U / eta
    (U - eta) (P'/P - gamma G'/G) = 3,
integrated inward from the strong-shock (Rankine-Hugoniot) values at
eta = 1: U = 2/(gamma+1), G = (gamma+1)/(gamma-1), P = 2/(gamma+1).  The
total energy E = 4 pi rho0 R^3 R'^2 I, I = int_0^1 eta^2 (G U^2/2 +
P/(gamma-1)) d eta, fixes xi0 = (25 / (16 pi I))^(1/5).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import solve_ivp


def _rhs(eta, y, gamma):
    U, G, P = y
    w = U - eta
    # rows: momentum, continuity, entropy; unknowns U', G', P'
    M = np.array([[w, 0.0, 1.0 / G],
                  [G, w, 0.0],
                  [0.0, -gamma * w / G, w / P]])
    b = np.array([1.5 * U, -2.0 * G * U / eta, 3.0])
    return np.linalg.solve(M, b)


def profile(gamma=5.0 / 3.0, eta_min=1e-4, n=4001):
    """eta (descending from 1), U, G, P of the similarity solution and xi0."""
    y1 = [2.0 / (gamma + 1.0), (gamma + 1.0) / (gamma - 1.0), 2.0 / (gamma + 1.0)]
    eta = np.concatenate([1.0 - np.logspace(-12, 0, n // 2) * (1.0 - 0.5),
                          np.geomspace(0.5, eta_min, n - n // 2)])
    eta = np.unique(np.clip(eta, eta_min, 1.0))[::-1]
    sol = solve_ivp(_rhs, (1.0, eta_min), y1, t_eval=eta, args=(gamma,), method="LSODA",
                    rtol=1e-10, atol=1e-13)
    if not sol.success:
        raise RuntimeError(sol.message)
    U, G, P = sol.y
    f = sol.t ** 2 * (0.5 * G * U * U + P / (gamma - 1.0))   # descending eta
    I = np.trapezoid(f[::-1], sol.t[::-1])
    xi0 = (25.0 / (16.0 * math.pi * I)) ** 0.2
    return sol.t, U, G, P, xi0


def solution(r, t, E=1.0, rho0=1.0, gamma=5.0 / 3.0):
    """Density, radial velocity and pressure at radii r and time t > 0."""
    eta_d, U, G, P, xi0 = profile(gamma)
    R = xi0 * (E * t * t / rho0) ** 0.2
    Rdot = 0.4 * R / t
    eta = np.asarray(r, dtype=np.float64) / R
    e, u_, g_, p_ = eta_d[::-1], U[::-1], G[::-1], P[::-1]   # ascending
    inside = eta < 1.0
    rho = np.where(inside, rho0 * np.interp(eta, e, g_), rho0)
    u = np.where(inside, Rdot * np.interp(eta, e, u_), 0.0)
    p = np.where(inside, rho0 * Rdot ** 2 * np.interp(eta, e, p_), 0.0)
    return rho, u, p, R
