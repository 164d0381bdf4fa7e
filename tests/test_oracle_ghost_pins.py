"""Pins of the oracle's ghost step (Omega, P, A; the text after Eq. (dudt))
and of the magnitude of its force and heating (Eq. (dvdt), (dudt)) against
facts fixed by thermodynamics and calculus rather than by re-typing the
formulas:

* d rho/dh and dN/dh equal the central finite differences of rho(h) and
  N(h) at fixed positions (Eq. (rho), (nneigh) evaluated at h(1 +- e));
* for equal masses the h of Eq. (nneigh) keeps rho h^3 fixed, so
  Omega = 1 + h/(3 rho) d rho/dh must equal h N'(h) / (3 N), with N'(h)
  from finite differences of a brute-force neighbour sum;
* adiabatic consistency: with equal masses, Eq. (dudt) must reproduce the
  first law du/dt = (P/rho^2) d rho/dt with P = (gamma - 1) rho u, where
  d rho/dt is the finite difference of the h-solved density along the
  particle trajectories x +- dt v.  A wrong Omega, gamma for gamma - 1 or a
  factor in A changes du/dt and fails;
* the acceleration amplitude of a perfect lattice with a sinusoidal
  internal energy equals the continuum -grad P / rho times a lattice factor
  R(k) that Taylor's theorem confines to [1 - (kh)^2/6, 1];
* energy conservation with random velocities then fixes the acceleration
  itself (sum m (du + v.a) = 0 for every v, with du/dt pinned above).

The last tests plant plausible mistakes in the oracle (monkeypatched on the
CPU) and check that these pins catch each one."""
import numpy as np
import pytest

from oracle import sph_oracle as O
import synth.configs as C
from tests.brute import all_pairs


def _wq(q):
    return np.where(q <= 0.5, 1 - 6 * q ** 2 + 6 * q ** 3, np.where(q <= 1, 2 * (1 - q) ** 3, 0.0))


def _equal_mass_box(seed=7, n=600):
    d = C.random_box(n, seed, "clumped", v_sigma=0.1)
    n = d["x"].shape[0]
    return d["x"], np.full(n, 1.0 / n), d["u"].astype(np.float64), d["v"].astype(np.float64)


def _adiabatic_error(x, m, u, v, dt=1e-5):
    """max_i |du_i/dt - (gamma-1) u_i/rho_i d rho_i/dt| / max |du/dt|."""
    f = O.evaluate(x, m, u, v=v, h_guess=0.2)
    rp = O.evaluate(x + dt * v, m, u, v=v, h_guess=f["h"])["rho"]
    rm = O.evaluate(x - dt * v, m, u, v=v, h_guess=f["h"])["rho"]
    drho_dt = (rp - rm) / (2 * dt)
    first_law = (O.GAMMA - 1.0) * u / f["rho"] * drho_dt
    return np.abs(first_law - f["dudt"]).max() / np.abs(f["dudt"]).max(), f


def _energy_error(x, m, u, v):
    f = O.evaluate(x, m, u, v=v, h_guess=0.2)
    e = m * (f["dudt"] + np.einsum("ij,ij->i", v, f["a"]))
    return abs(e.sum()) / np.abs(m * f["dudt"]).sum()


def _lattice_ratio(n_side=32, eps=0.01):
    """Fitted a_x amplitude over the continuum -(gamma-1) u0 eps k, and the
    Taylor lower bound 1 - (kh)^2/6 of the lattice factor."""
    d = C.perfect_lattice(n_side)
    k = 2 * np.pi
    x0 = d["x"][:, 0]
    u = 1.0 + eps * np.sin(k * x0)
    f = O.evaluate(d["x"], d["m"], u, h_guess=d["h_guess"])
    c = np.cos(k * x0)
    amp = (f["a"][:, 0] @ c) / (c @ c)
    resid = max(np.abs(f["a"][:, 0] - amp * c).max(), np.abs(f["a"][:, 1:]).max())
    cont = -(O.GAMMA - 1.0) * eps * k
    return amp / cont, 1.0 - (k * f["h"][0]) ** 2 / 6.0, resid / abs(amp)


def test_drho_dh_is_the_derivative_of_rho():
    d = C.random_box(500, 17, "clumped")
    m = d["m"].astype(np.float64)
    f = O.evaluate(d["x"], m, d["u"], h_guess=0.2)
    h, e = f["h"], 1e-6
    rp = O.density_at(f["nb"], m, h * (1 + e))["rho"]
    rm = O.density_at(f["nb"], m, h * (1 - e))["rho"]
    fd = (rp - rm) / (2 * e * h)
    assert np.allclose(f["drho_dh"], fd, rtol=1e-7, atol=1e-7 * np.abs(fd).max())


def test_dn_dh_is_the_derivative_of_the_neighbour_number():
    # the slope the h iteration steps with (Eq. (nneigh) differentiated in h)
    d = C.random_box(500, 19, "clumped")
    m = d["m"].astype(np.float64)
    f = O.evaluate(d["x"], m, d["u"], h_guess=0.2)
    h, e = f["h"], 1e-6
    npl = O.density_at(f["nb"], m, h * (1 + e))["nngb"]
    nmi = O.density_at(f["nb"], m, h * (1 - e))["nngb"]
    fd = (npl - nmi) / (2 * e * h)
    assert np.allclose(f["dnngb_dh"], fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())


def test_omega_equals_log_derivative_of_the_neighbour_number():
    x, m, u, v = _equal_mass_box()
    f = O.evaluate(x, m, u, h_guess=0.2)
    _, r = all_pairs(x)
    h, e = f["h"], 1e-6

    def N(hh):
        return 32.0 / 3.0 * _wq(r / hh[:, None]).sum(1)

    dN = (N(h * (1 + e)) - N(h * (1 - e))) / (2 * e * h)
    omega = h * dN / (3.0 * N(h))
    assert f["omega"].min() < 0.8 and f["omega"].max() > 1.2  # Omega far from 1 here
    assert np.allclose(f["omega"], omega, rtol=0, atol=1e-8)


def test_heating_obeys_the_first_law():
    err, f = _adiabatic_error(*_equal_mass_box())
    # the central difference of rho(t) is accurate to O(dt^2) ~ 1e-8 here
    assert err < 1e-6


def test_lattice_pressure_gradient_amplitude():
    R, lower, resid = _lattice_ratio()
    assert lower <= R <= 1.0 + 1e-9
    assert resid < 1e-9  # a pure cos(kx) response along x, nothing along y, z


def test_energy_conservation_with_equal_masses():
    assert _energy_error(*_equal_mass_box(seed=8)) < 1e-12


# ---- planted mistakes: each must fail one of the pins above ----------------
def _ghost_3h(h, rho, drho_dh, u, gamma=O.GAMMA):
    om = 1.0 + 3.0 * h * drho_dh / rho
    P = (gamma - 1.0) * rho * np.asarray(u, dtype=np.float64)
    return om, P, P / (om * rho * rho)


def _ghost_gamma(h, rho, drho_dh, u, gamma=O.GAMMA):
    om = 1.0 + h * drho_dh / (3.0 * rho)
    P = gamma * rho * np.asarray(u, dtype=np.float64)
    return om, P, P / (om * rho * rho)


def _ghost_no_omega(h, rho, drho_dh, u, gamma=O.GAMMA):
    om = 1.0 + h * drho_dh / (3.0 * rho)
    P = (gamma - 1.0) * rho * np.asarray(u, dtype=np.float64)
    return om, P, P / (rho * rho)


_force = O.force_from_pairs


def _force_twice(*args):
    a, du = _force(*args)
    return 2.0 * a, du


def _force_aj_twice(I, J, d, r, n, m, h, A, v):
    # the A_j term of Eq. (dvdt) doubled: a_i gains m_j A_j G_j once more
    a, du = _force(I, J, d, r, n, m, h, A, v)
    pos = r > 0
    I2, J2, d2, r2 = I[pos], J[pos], d[pos], r[pos]
    extra = -(np.asarray(m, dtype=np.float64)[J2] * A[J2] * O.G(r2, h[J2]))[:, None] * d2 / r2[:, None]
    a = a + np.stack([np.bincount(I2, weights=extra[:, k], minlength=n) for k in range(3)], axis=1)
    return a, du


@pytest.mark.parametrize("name,target,fake", [
    ("3h for h/3 in Omega", "ghost", _ghost_3h),
    ("gamma for gamma-1", "ghost", _ghost_gamma),
    ("Omega dropped from A", "ghost", _ghost_no_omega),
    ("factor 2 on the acceleration", "force_from_pairs", _force_twice),
    ("A_j term doubled", "force_from_pairs", _force_aj_twice),
])
def test_planted_mistakes_are_caught(monkeypatch, name, target, fake):
    monkeypatch.setattr(O, target, fake)
    box = _equal_mass_box()
    caught = []
    caught.append(_adiabatic_error(*box)[0] > 1e-3)
    caught.append(_energy_error(*_equal_mass_box(seed=8)) > 1e-6)
    R, lower, _ = _lattice_ratio(n_side=16)
    caught.append(not (lower <= R <= 1.0 + 1e-9))
    assert any(caught), name
