"""Exact solution of the one-dimensional Riemann problem for an ideal gas.

TEST INFRASTRUCTURE ONLY: the analytic reference for shock-tube runs (the
Sod-shock setup of Section 4.2 has two uniform states at rest).  Only
``tests/`` may use it; it shares no code with the CUDA library.

Method (the classical exact solver): the pressure p* between the two
nonlinear waves is the root of
    f(p) = f_L(p) + f_R(p) + (u_R - u_L) = 0,
where f_K is the velocity change across a shock (p > p_K, Rankine-Hugoniot)
or a rarefaction (p <= p_K, isentropic) into state K; f is monotone
increasing and concave, so Newton's method from below converges.  The
star velocity is u* = (u_L + u_R + f_R(p*) - f_L(p*)) / 2, and the solution
at a point depends on xi = (x - x0)/t only.
"""
from __future__ import annotations

import math

import numpy as np


def _f(p, rho, pk, ck, gamma):
    """Velocity jump across the wave into a state (rho, pk, sound speed ck)
    and its derivative in p."""
    if p > pk:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        q = math.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction
    e = (gamma - 1.0) / (2.0 * gamma)
    r = (p / pk) ** e
    return 2.0 * ck / (gamma - 1.0) * (r - 1.0), r / (rho * ck * (p / pk))


def star_state(rhoL, uL, pL, rhoR, uR, pR, gamma=5.0 / 3.0, tol=1e-14):
    """(p*, u*) of the Riemann problem."""
    cL = math.sqrt(gamma * pL / rhoL)
    cR = math.sqrt(gamma * pR / rhoR)
    if 2.0 * (cL + cR) / (gamma - 1.0) <= uR - uL:
        raise ValueError("the rarefactions create a vacuum")
    p = max(1e-12 * min(pL, pR), 0.5 * (pL + pR) - 0.125 * (uR - uL) * (rhoL + rhoR) * (cL + cR))
    for _ in range(200):
        fl, dl = _f(p, rhoL, pL, cL, gamma)
        fr, dr = _f(p, rhoR, pR, cR, gamma)
        F = fl + fr + (uR - uL)
        pn = p - F / (dl + dr)
        if pn <= 0.0:
            pn = 0.5 * p
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f(p, rhoL, pL, cL, gamma)
    fr, _ = _f(p, rhoR, pR, cR, gamma)
    return p, 0.5 * (uL + uR) + 0.5 * (fr - fl)


def sample(xi, rhoL, uL, pL, rhoR, uR, pR, gamma=5.0 / 3.0):
    """Density, velocity and pressure at xi = (x - x0)/t (arrays)."""
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    ps, us = star_state(rhoL, uL, pL, rhoR, uR, pR, gamma)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    out = np.empty((xi.size, 3))
    for k, s in enumerate(xi):
        if s <= us:  # left of the contact
            rho, u, p, c = rhoL, uL, pL, math.sqrt(gamma * pL / rhoL)
            if ps > p:  # left shock
                S = u - c * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / p + (gamma - 1.0) / (2.0 * gamma))
                out[k] = (rho, u, p) if s <= S else (rho * (ps / p + g1) / (g1 * ps / p + 1.0), us, ps)
            else:  # left rarefaction
                cs = c * (ps / p) ** ((gamma - 1.0) / (2.0 * gamma))
                head, tail = u - c, us - cs
                if s <= head:
                    out[k] = (rho, u, p)
                elif s >= tail:
                    out[k] = (rho * (ps / p) ** (1.0 / gamma), us, ps)
                else:
                    f = 2.0 / (gamma + 1.0) + g1 / c * (u - s)
                    out[k] = (rho * f ** (2.0 / (gamma - 1.0)),
                              2.0 / (gamma + 1.0) * (c + 0.5 * (gamma - 1.0) * u + s),
                              p * f ** (2.0 * gamma / (gamma - 1.0)))
        else:  # right of the contact, mirrored
            rho, u, p, c = rhoR, uR, pR, math.sqrt(gamma * pR / rhoR)
            if ps > p:  # right shock
                S = u + c * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / p + (gamma - 1.0) / (2.0 * gamma))
                out[k] = (rho, u, p) if s >= S else (rho * (ps / p + g1) / (g1 * ps / p + 1.0), us, ps)
            else:  # right rarefaction
                cs = c * (ps / p) ** ((gamma - 1.0) / (2.0 * gamma))
                head, tail = u + c, us + cs
                if s >= head:
                    out[k] = (rho, u, p)
                elif s <= tail:
                    out[k] = (rho * (ps / p) ** (1.0 / gamma), us, ps)
                else:
                    f = 2.0 / (gamma + 1.0) - g1 / c * (u - s)
                    out[k] = (rho * f ** (2.0 / (gamma - 1.0)),
                              2.0 / (gamma + 1.0) * (-c + 0.5 * (gamma - 1.0) * u + s),
                              p * f ** (2.0 * gamma / (gamma - 1.0)))
    return out[:, 0], out[:, 1], out[:, 2]
