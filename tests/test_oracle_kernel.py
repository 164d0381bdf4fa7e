"""Pins of the oracle's cubic-spline kernel (Section 2.1) against values
fixed by the printed formula and by mathematics: hand-evaluated rationals,
the unit normalisation, C^2 continuity at q = 1/2 and q = 1, and finite
differences of every derivative the oracle uses."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import sph_oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "kernel_values.json")


def test_kernel_values_from_printed_formula():
    data = json.load(open(GOLD))
    for row in data["w"]:
        q = float(Fraction(row["q"]))
        assert O.w(q) == pytest.approx(float(Fraction(row["w"])), abs=1e-15)


@pytest.mark.parametrize("h", [0.05, 1.0, 3.7])
def test_kernel_normalisation(h):
    val, err = quad(lambda r: 4 * math.pi * r * r * O.W(r, h), 0, h, points=[0.5 * h],
                    epsabs=1e-14, epsrel=1e-13)
    assert val == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("q0", [0.5, 1.0])
def test_kernel_c2_continuity(q0):
    e = 1e-9
    for f, tol in ((O.w, 1e-8), (O.dw, 1e-7), (O.d2w, 1e-7)):
        assert abs(float(f(q0 - e)) - float(f(q0 + e))) < tol


def _fd(f, x, eps):
    return (f(x + eps) - f(x - eps)) / (2 * eps)


def test_kernel_derivatives_finite_difference():
    q = np.linspace(0.013, 0.987, 101)
    q = q[np.abs(q - 0.5) > 1e-3]
    assert np.allclose(_fd(O.w, q, 1e-6), O.dw(q), atol=1e-8)
    assert np.allclose(_fd(O.dw, q, 1e-6), O.d2w(q), atol=1e-7)
    r, h = 0.37 * q, 0.37
    assert np.allclose(_fd(lambda hh: O.W(r, hh), h, 1e-7), O.dW_dh(r, h), rtol=1e-6, atol=1e-6)
    assert np.allclose(_fd(lambda rr: O.W(rr, h), r, 1e-7), O.G(r, h), rtol=1e-6, atol=1e-6)
    assert np.allclose(_fd(lambda rr: O.G(rr, h), r, 1e-7), O.dG_dr(r, h), rtol=1e-6, atol=1e-5)
    assert np.allclose(_fd(lambda hh: O.G(r, hh), h, 1e-7), O.dG_dh(r, h), rtol=1e-6, atol=1e-5)
    assert np.allclose(_fd(lambda hh: O.dW_dh(r, hh), h, 1e-7), O.d2W_dh2(r, h), rtol=1e-6, atol=1e-5)


def test_gradient_sign_is_repulsive():
    # grad_i W = G(r) (x_i - x_j)/r with G = dW/dr <= 0 inside the support
    q = np.linspace(0.01, 0.99, 50)
    assert np.all(O.G(q, 1.0) < 0)
