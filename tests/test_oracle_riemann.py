"""Pins of the exact Riemann solver (the analytic reference of the
Sod-shock setup, Section 4.2) by the conservation laws and invariants the
solution must satisfy, not by tabulated values: Rankine-Hugoniot jump
conditions across the shock, continuity of pressure and velocity across the
contact, isentropy and the Riemann invariant through the rarefaction, the
far-field states, and mirror symmetry."""
import math

import numpy as np
import pytest

from oracle import riemann as R

G = 5.0 / 3.0
# the paper's shock tube (both states at rest) and a mirrored, moving variant
CASES = [(4.0, 0.0, 1.0, 1.0, 0.0, 0.1795), (1.0, 0.3, 0.1795, 4.0, 0.3, 1.0),
         (1.0, 0.0, 1.0, 0.125, 0.0, 0.1)]


def _fluxes(rho, u, p, s):
    """Mass, momentum and energy fluxes in the frame moving with speed s."""
    w = u - s
    E = p / (G - 1.0) + 0.5 * rho * w * w
    return np.array([rho * w, rho * w * w + p, (E + p) * w])


@pytest.mark.parametrize("case", CASES)
def test_jump_conditions_and_invariants(case):
    rL, uL, pL, rR, uR, pR = case
    ps, us = R.star_state(*case, gamma=G)
    assert min(pL, pR) < ps < max(pL, pR)       # one shock, one rarefaction here
    xi = np.linspace(-3, 3, 60001)
    rho, u, p = R.sample(xi, *case, gamma=G)
    # far field
    assert (rho[0], u[0], p[0]) == (rL, uL, pL) and (rho[-1], u[-1], p[-1]) == (rR, uR, pR)
    # the shock: the only jump of pressure (the contact carries none)
    k = int(np.argmax(np.abs(np.diff(p))))
    S = 0.5 * (xi[k] + xi[k + 1])
    a, b = (k - 2, k + 3)
    fa, fb = _fluxes(rho[a], u[a], p[a], S), _fluxes(rho[b], u[b], p[b], S)
    assert np.allclose(fa, fb, rtol=2e-3, atol=2e-3 * np.abs(fa).max())
    # pressure and velocity are continuous everywhere except at the shock
    jump = np.ones(xi.size - 1, bool)
    jump[max(k - 1, 0):k + 2] = False
    assert np.abs(np.diff(p))[jump].max() < 1e-3 * max(pL, pR)
    assert np.abs(np.diff(u))[jump].max() < 1e-3 * (abs(us) + 1.0)
    # the star region has p = p*, u = u* on both sides of the contact
    near = np.abs(xi - us) < 1e-3
    assert np.allclose(p[near], ps) and np.allclose(u[near], us)
    # the rarefaction is isentropic and keeps its Riemann invariant
    left_high = pL > pR
    rho0, u0, p0 = (rL, uL, pL) if left_high else (rR, uR, pR)
    c = np.sqrt(G * p / rho)
    fan = (p < p0 * (1 - 1e-9)) & (p > ps * (1 + 1e-9))
    assert fan.sum() > 100
    np.testing.assert_allclose(p[fan] / rho[fan] ** G, p0 / rho0 ** G, rtol=1e-10)
    c0 = math.sqrt(G * p0 / rho0)
    inv = u[fan] + (2 * c[fan] / (G - 1) if left_high else -2 * c[fan] / (G - 1))
    np.testing.assert_allclose(inv, u0 + (2 * c0 / (G - 1) if left_high else -2 * c0 / (G - 1)),
                               rtol=1e-10, atol=1e-12)


def test_mirror_symmetry():
    a = (4.0, 0.2, 1.0, 1.0, -0.1, 0.1795)
    b = (1.0, 0.1, 0.1795, 4.0, -0.2, 1.0)       # x -> -x
    xi = np.linspace(-2, 2, 401)
    ra, ua, pa = R.sample(xi, *a, gamma=G)
    rb, ub, pb = R.sample(-xi, *b, gamma=G)
    np.testing.assert_allclose(ra, rb, rtol=1e-12)
    np.testing.assert_allclose(ua, -ub, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(pa, pb, rtol=1e-12)


def test_equal_states_and_vacuum():
    rho, u, p = R.sample(np.linspace(-1, 1, 11), 1.0, 0.2, 1.0, 1.0, 0.2, 1.0, gamma=G)
    assert np.all(rho == 1.0) and np.allclose(u, 0.2) and np.allclose(p, 1.0)
    with pytest.raises(ValueError):
        R.star_state(1.0, -10.0, 0.1, 1.0, 10.0, 0.1, gamma=G)
