"""Pins of the Sedov-Taylor similarity solution (the analytic reference of
the Sedov-blast setup, Section 4.2) by properties the equations fix but the
integration does not impose: mass conservation (the swept-up gas is all
inside the shock), the central asymptotics U/eta -> 1/gamma,
G ~ eta^(3/(gamma-1)) and a pressure plateau (from the leading-order
balance of the similarity equations), the released energy recovered
from the dimensional solution, and the published shock-radius constants."""
import math

import numpy as np
import pytest

from oracle import sedov as S


@pytest.mark.parametrize("gamma", [5.0 / 3.0, 1.4])
def test_mass_and_central_asymptotics(gamma):
    eta, U, G, P, xi0 = S.profile(gamma)
    x, g = eta[::-1], G[::-1]
    assert abs(np.trapezoid(x * x * g, x) - 1.0 / 3.0) < 2e-4
    def at(e):
        k = int(np.argmin(np.abs(eta - e)))
        return eta[k], U[k], G[k], P[k]
    e1, u1, g1, p1 = at(0.2)      # G stays far above the integrator's tolerance
    e2, u2, g2, p2 = at(0.1)
    assert abs(u1 / e1 - 1.0 / gamma) < 1e-3 and abs(u2 / e2 - 1.0 / gamma) < 1e-3
    slope = math.log(g1 / g2) / math.log(e1 / e2)
    assert abs(slope - 3.0 / (gamma - 1.0)) < 2e-2
    assert abs(p1 / p2 - 1.0) < 1e-3
    assert 0.9 < xi0 < 1.4


def test_energy_of_the_dimensional_solution():
    E, rho0, t = 2.0, 0.5, 0.3
    r = np.linspace(0.0, 3.0, 200001)
    rho, u, p, R = S.solution(r, t, E=E, rho0=rho0)
    assert 0 < R < 3.0
    e = (0.5 * rho * u * u + p / (2.0 / 3.0)) * 4.0 * math.pi * r * r
    assert abs(np.trapezoid(e, r) / E - 1.0) < 2e-3
    # the shocked shell holds the swept-up mass
    inside = r < R
    m = np.trapezoid((rho * 4.0 * math.pi * r * r)[inside], r[inside])
    assert abs(m / (4.0 / 3.0 * math.pi * R ** 3 * rho0) - 1.0) < 2e-3


@pytest.mark.parametrize("gamma,alpha", [(1.4, 0.851), (5.0 / 3.0, 0.4936)])
def test_xi0_matches_the_published_energy_constants(gamma, alpha):
    # Sedov's energy integral alpha, tabulated for the spherical blast
    # (Sedov, "Similarity and Dimensional Methods in Mechanics", 1959;
    # Taylor, Proc. R. Soc. A 201, 1950, for gamma = 1.4), gives
    # R = (E t^2 / (alpha rho0))^(1/5), i.e. xi0 = alpha^(-1/5).  The
    # tabulated alpha carries 3-4 significant digits.
    xi0 = S.profile(gamma)[4]
    assert abs(xi0 / alpha ** -0.2 - 1.0) < 5e-4
