"""Pins of the oracle's velocity-Verlet step (Section 4.1): exact momentum
conservation, the total energy error positive and of third order in the
step for inviscid flow, viscous runs converging too, and a uniform lattice
at rest staying at rest."""
import numpy as np

from oracle import sph_oracle as O
import synth.configs as C


def _run(d, dt, steps, alpha):
    x, v, u = d["x"].astype(np.float64), d["v"].astype(np.float64), d["u"].astype(np.float64)
    m = d["m"].astype(np.float64)
    h = 0.1
    for _ in range(steps):
        x, v, u, h = O.verlet_step(x, v, u, m, dt, h, alpha=alpha)
    return x, v, u


def _energy(m, v, u):
    return float(np.sum(m * (0.5 * np.sum(v * v, axis=1) + u)))


def test_momentum_exact_and_energy_error_order():
    d = C.random_box(1500, 31, "clumped", v_sigma=0.2)
    m = d["m"].astype(np.float64)
    v0 = d["v"].astype(np.float64)
    e0 = _energy(m, v0, d["u"].astype(np.float64))
    T = 0.004
    for alpha in (0.0, 0.8):
        errs = []
        for steps in (2, 4):
            x, v, u = _run(d, T / steps, steps, alpha=alpha)
            p0, p1 = (m[:, None] * v0).sum(0), (m[:, None] * v).sum(0)
            assert np.abs(p1 - p0).max() <= 1e-12 * np.abs(m[:, None] * v).sum()
            errs.append(_energy(m, v, u) - e0)
        if alpha == 0.0:
            # dt^2/8 sum m |a(t+dt) - a(t)|^2 per step: positive, third order
            assert errs[0] > 0 and errs[1] > 0 and errs[1] < errs[0] / 5.0
        else:
            assert abs(errs[1]) < abs(errs[0]) / 2.0


def test_lattice_at_rest_stays_at_rest():
    d = C.perfect_lattice(8)
    n = d["x"].shape[0]
    d = dict(d, v=np.zeros((n, 3), np.float32))
    x, v, u = _run(d, 0.01, 2, alpha=0.8)
    assert np.abs(v).max() <= 1e-12
    np.testing.assert_allclose(x, d["x"], atol=1e-14)
    np.testing.assert_allclose(u, d["u"], rtol=1e-14)
