"""Pins of the oracle's artificial viscosity, Balsara switch, velocity
derivatives and time-step criterion (Section 4.1, Eq. (dt)) by conservation
laws, Galilean invariance, exact symmetry zeros of linear velocity fields
and the cubic symmetry of a perfect lattice -- none of them a retyping of
the formulas."""
import numpy as np
import pytest

from oracle import sph_oracle as O
import synth.configs as C

ALPHA, CCFL = 0.8, 0.25


@pytest.fixture(scope="module")
def lattice():
    d = C.perfect_lattice(16)   # spacing 2^-4: every site exact, the lattice exactly cubic
    a = 1.0 / 16
    h = np.full(d["x"].shape[0], 2.251490 * a)
    fwd = O.evaluate(d["x"], d["m"], d["u"], h=h)
    # particles whose neighbourhood stays clear of the periodic faces, where
    # a global linear velocity field is continuous
    c = d["x"] - 0.5
    interior = np.all(np.abs(c) < 0.5 - 1.05 * h[0], axis=1)
    assert interior.sum() >= 64
    return d, fwd, c, interior, h[0]


@pytest.fixture(scope="module")
def clumped():
    d = C.random_box(3000, 21, "clumped", v_sigma=0.3)
    fwd = O.evaluate(d["x"], d["m"], d["u"], v=d["v"], h_guess=0.1)
    return d, fwd


def test_viscosity_conserves_momentum_and_energy_and_only_heats(clumped):
    d, fwd = clumped
    vis = O.evaluate_viscosity(fwd, d["x"], d["m"], d["u"], d["v"], ALPHA, CCFL)
    m = d["m"].astype(np.float64)
    v = d["v"].astype(np.float64)
    ma = m[:, None] * vis["a_visc"]
    assert np.abs(ma.sum(0)).max() <= 1e-12 * np.abs(ma).sum()
    # sum_i m_i (du_i + v_i . a_i) = 0: the viscous work goes into heat
    e = m * (vis["dudt_visc"] + np.einsum("ij,ij->i", v, vis["a_visc"]))
    assert abs(e.sum()) <= 1e-12 * np.abs(e).sum()
    # every pair term of the heating is >= 0, so is every particle's
    assert vis["dudt_visc"].min() >= 0.0
    assert vis["dudt_visc"].sum() > 0.0
    assert np.all((vis["balsara"] >= 0) & (vis["balsara"] <= 1))


def test_no_relative_motion_no_viscosity(clumped):
    d, fwd = clumped
    n = d["x"].shape[0]
    dts = []
    for v in (np.zeros((n, 3)), np.tile([0.3, -1.2, 2.0], (n, 1))):   # rest, uniform drift
        vis = O.evaluate_viscosity(fwd, d["x"], d["m"], d["u"], v, ALPHA, CCFL)
        assert np.abs(vis["a_visc"]).max() == 0.0 and np.abs(vis["dudt_visc"]).max() == 0.0
        assert np.abs(vis["div"]).max() <= 1e-12 and np.abs(vis["curl"]).max() <= 1e-12
        dts.append(vis["dt"])
    # Galilean invariance, and without approaching pairs the signal speed is
    # a sum of two sound speeds of the box
    assert np.array_equal(dts[0], dts[1])
    c = O.sound_speed(d["u"])
    h = fwd["h"]
    assert np.all(dts[0] >= CCFL * 2 * h / (c + c.max()) * (1 - 1e-12))
    assert np.all(dts[0] <= CCFL * 2 * h / (c + c.min()) * (1 + 1e-12))


def test_static_uniform_medium_time_step(lattice):
    d, fwd, c, interior, h = lattice
    n = d["x"].shape[0]
    vis = O.evaluate_viscosity(fwd, d["x"], d["m"], d["u"], np.zeros((n, 3)), ALPHA, CCFL)
    cs = O.sound_speed(d["u"])
    np.testing.assert_allclose(vis["dt"], CCFL * h / cs, rtol=1e-14)


def test_expansion_rotation_shear_on_a_perfect_lattice(lattice):
    d, fwd, c, interior, h = lattice
    lam, om, s = 0.7, np.array([0.0, 0.0, 1.3]), 0.9
    ex = O.evaluate_viscosity(fwd, d["x"], d["m"], d["u"], lam * c, ALPHA, CCFL)
    rot = O.evaluate_viscosity(fwd, d["x"], d["m"], d["u"], np.cross(om, c), ALPHA, CCFL)
    sh = O.evaluate_viscosity(fwd, d["x"], d["m"], d["u"],
                              np.stack([s * c[:, 1], 0 * c[:, 0], 0 * c[:, 0]], axis=1), ALPHA, CCFL)
    I = interior
    # a pure expansion has no curl, a rigid rotation no divergence (exact
    # for any arrangement: parallel vectors in the cross / triple products)
    assert np.abs(ex["curl"][I]).max() <= 1e-12 * np.abs(ex["div"][I]).max()
    assert np.abs(rot["div"][I]).max() <= 1e-12 * np.abs(rot["curl"][I]).max()
    # cubic symmetry: div(lam x) = 3 lam k and curl(om x x) = 2 om k with
    # the same lattice factor k, as for the exact derivatives (sign included)
    k = ex["div"][I] / (3 * lam)
    np.testing.assert_allclose(rot["curl"][I], 2 * om[None, :] * k[:, None], rtol=1e-10,
                               atol=1e-12 * abs(k).max())
    assert np.all(k > 0)
    # Balsara: on in compression/expansion, off in rotation and in shear
    assert np.all(ex["balsara"][I] > 0.99)
    assert np.abs(rot["balsara"][I]).max() <= 1e-12
    assert np.abs(sh["div"][I]).max() <= 1e-12 * np.abs(sh["curl"][I]).max()
    assert np.abs(sh["balsara"][I]).max() <= 1e-12
    # receding pairs feel no viscosity: an expansion is inviscid, and only a
    # compression heats and shortens the time step
    assert np.abs(ex["a_visc"][I]).max() == 0.0 and np.abs(ex["dudt_visc"][I]).max() == 0.0
    cs = O.sound_speed(d["u"])
    np.testing.assert_allclose(ex["dt"][I], CCFL * h / cs[I], rtol=1e-14)
    co = O.evaluate_viscosity(fwd, d["x"], d["m"], d["u"], -lam * c, ALPHA, CCFL)
    assert np.all(co["dudt_visc"][I] > 0) and np.all(co["dt"][I] < CCFL * h / cs[I])
    # the compression's viscous force vanishes by symmetry (equal and
    # opposite neighbours with equal switches) where the neighbours are
    # interior too; the heating is uniform there
    D = np.all(np.abs(c) < 0.5 - 2.1 * h, axis=1)
    assert D.sum() >= 27
    assert np.abs(co["a_visc"][D]).max() <= 1e-10 * np.abs(co["dudt_visc"][D]).max()
    np.testing.assert_allclose(co["dudt_visc"][D], co["dudt_visc"][D].mean(), rtol=1e-10)
