"""Pins of the oracle against what the paper and mathematics fix:
perfect-lattice closed forms (Eq. (rho), Eq. (nneigh)), O(N^2) brute
force, the equal-mass identity rho = 36 m/(pi h^3) at N_ngb = 48,
momentum and energy conservation of Eq. (dvdt)/(dudt), the physical sign
of the pressure force and of compressional heating, and finite
differences of the reverse-mode gradient."""
import math

import numpy as np
import pytest

from oracle import sph_oracle as O
import synth.configs as C
from tests.brute import all_pairs, directed_sets, lattice_nngb


def _lattice_root():
    lo, hi = 1.5, 3.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if lattice_nngb(mid)[0] < 48.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def test_perfect_lattice_closed_form():
    root = _lattice_root()
    assert root == pytest.approx(2.251490, abs=5e-7)
    _, count, rr = lattice_nngb(root)
    assert count == 57
    d = C.perfect_lattice(16)  # a = 1/16: sites exact after 2^-24 quantisation
    a = 1.0 / 16
    f = O.evaluate(d["x"], d["m"], d["u"], h_guess=d["h_guess"])
    assert np.allclose(f["h"] / a, root, rtol=1e-11, atol=0)
    assert np.all(f["count"] == 57)
    m = float(d["m"][0])
    # rho = m sum_n W(|n| a, h) on the lattice
    rho_lat = m * 8 / (math.pi * (root * a) ** 3) * np.sum(
        np.where(rr <= 0.5, 1 - 6 * rr ** 2 + 6 * rr ** 3, np.where(rr <= 1, 2 * (1 - rr) ** 3, 0)))
    assert np.allclose(f["rho"], rho_lat, rtol=1e-11)
    assert f["rho"][0] * a ** 3 / m == pytest.approx(1.004021, abs=2e-6)
    # symmetric neighbourhood: no net force
    assert np.abs(f["a"]).max() < 1e-10 * np.abs(f["A"]).max() * m / a ** 4


@pytest.mark.parametrize("kind,seed", [("uniform", 11), ("clumped", 12), ("lattice", 13)])
def test_oracle_matches_brute_force(kind, seed):
    d = C.random_box(500, seed, kind)
    x, m = d["x"], d["m"].astype(np.float64)
    f = O.evaluate(x, m, d["u"], h_guess=0.2)
    h = f["h"]
    S, r = directed_sets(x, h)
    # pair sets
    i, j, _, _ = O.directed_pairs(f["nb"], h)
    mine = np.zeros_like(S)
    mine[i, j] = True
    assert np.array_equal(mine, S)
    # N(h) = 48 checked by brute force at the oracle's h
    q = np.where(S, r / h[:, None], 2.0)
    wq = np.where(q <= 0.5, 1 - 6 * q ** 2 + 6 * q ** 3, np.where(q <= 1, 2 * (1 - q) ** 3, 0))
    assert np.allclose(32 / 3 * wq.sum(1), 48.0, rtol=0, atol=1e-10)
    rho = (m[None, :] * 8 / (math.pi * h[:, None] ** 3) * wq).sum(1)
    assert np.allclose(f["rho"], rho, rtol=1e-12)
    # force pair set r < max(h_i, h_j)
    I, J, _, _ = O.force_pairs_all(f["nb"], h)
    F = np.zeros_like(S)
    F[I, J] = True
    ref = (S | S.T)
    np.fill_diagonal(ref, False)
    assert np.array_equal(F, ref)


def test_equal_mass_density_identity():
    d = C.uniform_lattice(10, seed=5)
    f = O.evaluate(d["x"], d["m"], d["u"], h_guess=d["h_guess"])
    m = float(d["m"][0])
    assert np.allclose(f["rho"], 36 * m / (math.pi * f["h"] ** 3), rtol=1e-12)


@pytest.mark.parametrize("seed", [21, 22])
def test_momentum_and_energy_conservation(seed):
    d = C.random_box(700, seed, "clumped", v_sigma=0.1)
    m = d["m"].astype(np.float64)
    v = d["v"].astype(np.float64)
    f = O.evaluate(d["x"], m, d["u"], v=v, h_guess=0.2)
    ma = m[:, None] * f["a"]
    assert np.abs(ma.sum(0)).max() < 1e-13 * np.abs(ma).sum()
    e = m * (f["dudt"] + np.einsum("ij,ij->i", v, f["a"]))
    assert abs(e.sum()) < 1e-12 * np.abs(e).sum() + 1e-12 * np.abs(m * f["dudt"]).sum()


def test_pressure_force_points_down_the_gradient():
    d = C.sinusoid(16, seed=4)
    f = O.evaluate(d["x"], d["m"], np.ones(d["x"].shape[0], np.float32), h_guess=2.25 / 16)
    # u = 1: P ~ rho ~ 1 + 0.3 sin(2 pi x); acceleration ~ -grad P / rho ~ -cos(2 pi x)
    c = np.corrcoef(f["a"][:, 0], -np.cos(2 * np.pi * d["x"][:, 0]))[0, 1]
    assert c > 0.5  # a flipped sign gives a strongly negative correlation


def test_compression_heats():
    d = C.uniform_lattice(12, seed=6)
    n = d["x"].shape[0]
    v = np.zeros((n, 3))
    v[:, 0] = -0.1 * np.sin(2 * np.pi * d["x"][:, 0])  # converging on x = 0
    f = O.evaluate(d["x"], d["m"], d["u"], v=v, h_guess=d["h_guess"])
    c = np.corrcoef(f["dudt"], np.cos(2 * np.pi * d["x"][:, 0]))[0, 1]
    assert c > 0.5  # a flipped sign gives a strongly negative correlation


def test_gradient_matches_central_differences():
    d = C.random_box(400, 31, "clumped", v_sigma=0.1)
    x, m, u, v = d["x"], d["m"].astype(float), d["u"].astype(float), d["v"].astype(float)
    rng = np.random.default_rng(3)
    n = x.shape[0]
    gr, ga, gdu = rng.normal(size=n), rng.normal(size=(n, 3)), rng.normal(size=n)

    def L(x, m, u):
        f = O.evaluate(x, m, u, v=v, h_guess=0.2)
        return (gr * f["rho"]).sum() + (ga * f["a"]).sum() + (gdu * f["dudt"]).sum(), f

    _, f = L(x, m, u)
    g = O.gradient(f, x, m, u, v, gr, ga, gdu)
    for _ in range(4):
        i, c = rng.integers(n), rng.integers(3)
        xp, xm = x.copy(), x.copy()
        xp[i, c] += 1e-6
        xm[i, c] -= 1e-6
        fd = (L(xp, m, u)[0] - L(xm, m, u)[0]) / 2e-6
        assert g["g_x"][i, c] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(g["g_x"]).max())
    for _ in range(3):
        i = rng.integers(n)
        e = 1e-6 * m[i]
        mp, mm = m.copy(), m.copy()
        mp[i] += e
        mm[i] -= e
        fd = (L(x, mp, u)[0] - L(x, mm, u)[0]) / (2 * e)
        assert g["g_m"][i] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(g["g_m"]).max())
        up, um = u.copy(), u.copy()
        up[i] += 1e-6
        um[i] -= 1e-6
        fd = (L(x, m, up)[0] - L(x, m, um)[0]) / 2e-6
        assert g["g_u"][i] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(g["g_u"]).max())


def test_sampled_evaluation_matches_full():
    d = C.random_box(3000, 41, "clumped")
    full = O.evaluate(d["x"], d["m"], d["u"], h_guess=0.15)
    s = np.sort(np.random.default_rng(0).choice(3000, 200, replace=False))
    smp = O.evaluate_sample(d["x"], d["m"], d["u"], s)
    for k in ("h", "rho", "omega", "dudt", "nngb"):
        assert np.allclose(smp[k], full[k][s], rtol=1e-11, atol=1e-12), k
    assert np.allclose(smp["a"], full["a"][s], rtol=1e-10, atol=1e-10 * np.abs(full["a"]).max())
    assert np.array_equal(smp["count"], full["count"][s])
    assert np.array_equal(smp["force_count"], full["force_count"][s])
