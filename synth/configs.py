"""Seeded synthetic particle sets for the SPH density/force path.

This module only draws inputs: positions, masses, internal energies,
velocities and smoothing-length guesses.  It holds none of the SPH
arithmetic (no kernel, no density, no force), so both the FP64 oracle and
the CUDA path can take their inputs from here without sharing any of the
method's code.

All positions live in a periodic cube [0, L)^3 with L = 1 and are
quantised to multiples of 2^-24 (``quantise``) so that every cell-relative
coordinate and every coordinate difference of neighbouring particles is
exact in FP32.  Masses and energies are returned as float32 arrays because
those are the values the GPU receives; the oracle widens the same float32
values to float64.

Workload recipes (one function each):
  * ``uniform_lattice``  16^3 jittered lattice, equal masses (the small
    parity case).
  * ``multires``         128^3 particles: a jittered lattice with 20 % of
    its sites removed plus a central Plummer clump holding 20 % of the
    particles (h spans about 100x); energies log-uniform over 2 decades.
  * ``batch_boxes``      64 independent boxes of 5k..500k particles
    (log-uniform), half uniform and half in Gaussian clumps.
  * ``sinusoid``         64^3 lattice whose x coordinate follows the
    inverse CDF of rho ~ 1 + 0.3 sin(2 pi x), jittered; u = 1 + 0.5 sin 2 pi y.
  * ``zeldovich``        256^3 lattice displaced by a Gaussian random field
    with P(k) ~ k^-2 (cosmology-like clustering).
  * ``lognormal``        256^3 particles sampled from the log-normal density
    exp(sigma G) of the same kind of Gaussian field G (h spans ~10^3).
"""
from __future__ import annotations

import numpy as np

Q24 = float(2 ** 24)


def quantise(x: np.ndarray, box: float = 1.0) -> np.ndarray:
    """Round positions to multiples of box*2^-24 and wrap them into [0, box)."""
    q = np.rint(np.asarray(x, dtype=np.float64) / box * Q24)
    q = np.mod(q, Q24)
    return q * (box / Q24)


def _jittered_lattice(n_side: int, jitter: float, rng: np.random.Generator) -> np.ndarray:
    a = 1.0 / n_side
    g = (np.arange(n_side) + 0.5) * a
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    x = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    if jitter > 0:
        x = x + rng.uniform(-jitter * a, jitter * a, size=x.shape)
    return x


def _pack(x, m, u, v=None, h_guess=None, name="", **extra):
    n = x.shape[0]
    if v is None:
        v = np.zeros((n, 3), dtype=np.float32)
    d = dict(
        name=name,
        x=quantise(x),
        m=np.asarray(m, dtype=np.float32).reshape(n),
        u=np.asarray(u, dtype=np.float32).reshape(n),
        v=np.asarray(v, dtype=np.float32).reshape(n, 3),
        h_guess=None if h_guess is None else np.asarray(h_guess, dtype=np.float32).reshape(n),
        box=1.0,
    )
    d.update(extra)
    return d


def uniform_lattice(n_side: int = 16, seed: int = 1, jitter: float = 0.1) -> dict:
    """Jittered cubic lattice: spacing a = 1/n_side, sites at (i + 1/2) a,
    each component displaced by U(-jitter a, jitter a); m = 1/N, u = 1,
    v = 0, h_guess = 2.2515 a (the perfect-lattice root of N_ngb = 48)."""
    rng = np.random.default_rng(seed)
    x = _jittered_lattice(n_side, jitter, rng)
    n = x.shape[0]
    a = 1.0 / n_side
    return _pack(x, np.full(n, 1.0 / n), np.ones(n), h_guess=np.full(n, 2.2515 * a),
                 name=f"uniform_lattice_{n_side}^3")


def perfect_lattice(n_side: int = 16) -> dict:
    """Unjittered cubic lattice (closed-form test case)."""
    x = _jittered_lattice(n_side, 0.0, np.random.default_rng(0))
    n = x.shape[0]
    a = 1.0 / n_side
    return _pack(x, np.full(n, 1.0 / n), np.ones(n), h_guess=np.full(n, 2.2515 * a),
                 name=f"perfect_lattice_{n_side}^3")


def _plummer(n: int, b: float, rmax: float, center, rng: np.random.Generator) -> np.ndarray:
    """Plummer sphere sample: r = b / sqrt(U^(-2/3) - 1), truncated at rmax
    by resampling, isotropic directions."""
    r = np.empty(0)
    while r.size < n:
        U = rng.uniform(0.0, 1.0, size=2 * (n - r.size) + 16)
        U = U[U > 0]
        rr = b / np.sqrt(U ** (-2.0 / 3.0) - 1.0)
        r = np.concatenate([r, rr[rr <= rmax]])
    r = r[:n]
    mu = rng.uniform(-1.0, 1.0, size=n)
    phi = rng.uniform(0.0, 2 * np.pi, size=n)
    s = np.sqrt(1 - mu * mu)
    d = np.stack([s * np.cos(phi), s * np.sin(phi), mu], axis=1)
    return np.asarray(center)[None, :] + r[:, None] * d


def multires(n_side: int = 128, seed: int = 2, clump_frac: float = 0.2,
             removed_frac: float = 0.2, b: float = 0.004, rmax: float = 0.3) -> dict:
    """Multi-resolution box: a jittered n_side^3 lattice (+-0.1 a) with a
    seeded random ``removed_frac`` of its sites removed, plus a Plummer clump
    (scale b, truncated at rmax) centred at (1/2, 1/2, 1/2) holding the
    remaining particles so that the total is n_side^3.  m = 1/N,
    u = 10^U(-1, 1), v = 0."""
    rng = np.random.default_rng(seed)
    n = n_side ** 3
    lat = _jittered_lattice(n_side, 0.1, rng)
    n_removed = int(round(removed_frac * n))
    keep = np.ones(n, dtype=bool)
    keep[rng.choice(n, size=n_removed, replace=False)] = False
    lat = lat[keep]
    n_clump = n - lat.shape[0]
    clump = _plummer(n_clump, b, rmax, (0.5, 0.5, 0.5), rng)
    x = np.concatenate([lat, clump], axis=0)
    u = 10.0 ** rng.uniform(-1.0, 1.0, size=n)
    return _pack(x, np.full(n, 1.0 / n), u, name=f"multires_{n_side}^3",
                 clump_count=n_clump)


def concat_boxes(boxes: list[dict]) -> dict:
    """Concatenate independent unit boxes for a batched build: positions,
    masses, energies, velocities back to back, with the particle offsets."""
    off = np.concatenate([[0], np.cumsum([b["x"].shape[0] for b in boxes])]).astype(np.int64)
    return dict(name=f"batch{len(boxes)}", x=np.concatenate([b["x"] for b in boxes]),
                m=np.concatenate([b["m"] for b in boxes]), u=np.concatenate([b["u"] for b in boxes]),
                v=np.concatenate([b["v"] for b in boxes]), h_guess=None, box=1.0,
                offsets=off, boxes=[1.0] * len(boxes))


def batch_boxes(nbox: int = 64, seed: int = 3, nmin: float = 5e3, nmax: float = 5e5,
                sigma: float = 0.03) -> list[dict]:
    """Independent periodic boxes.  Box b draws N_b = round(exp U(ln nmin,
    ln nmax)) with its own generator (seed + b): half the particles uniform,
    half in 1 + (b mod 4) Gaussian clumps of width sigma at uniform centres,
    wrapped.  m = 1/N_b, u = 1, v = 0."""
    boxes = []
    for b in range(nbox):
        rng = np.random.default_rng(seed + b)
        nb = int(round(np.exp(rng.uniform(np.log(nmin), np.log(nmax)))))
        n_uni = nb // 2
        n_cl = nb - n_uni
        xu = rng.uniform(0.0, 1.0, size=(n_uni, 3))
        k = 1 + (b % 4)
        centres = rng.uniform(0.0, 1.0, size=(k, 3))
        which = rng.integers(0, k, size=n_cl)
        xc = centres[which] + rng.normal(0.0, sigma, size=(n_cl, 3))
        x = np.concatenate([xu, xc], axis=0)
        boxes.append(_pack(x, np.full(nb, 1.0 / nb), np.ones(nb), name=f"box{b}_{nb}"))
    return boxes


def sinusoid(n_side: int = 64, seed: int = 4, amp: float = 0.3) -> dict:
    """x from the inverse CDF of rho ~ 1 + amp sin(2 pi x): solve
    x + amp (1 - cos 2 pi x) / (2 pi) = q at q = (i + 1/2)/n_side by
    bisection; y, z on the lattice; every component then jittered by
    U(-0.1 a, 0.1 a).  m = 1/N, u = 1 + 0.5 sin(2 pi y), v = 0."""
    rng = np.random.default_rng(seed)
    a = 1.0 / n_side
    q = (np.arange(n_side) + 0.5) * a
    lo = np.zeros_like(q)
    hi = np.ones_like(q)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        f = mid + amp * (1.0 - np.cos(2 * np.pi * mid)) / (2 * np.pi) - q
        lo = np.where(f < 0, mid, lo)
        hi = np.where(f < 0, hi, mid)
    gx = 0.5 * (lo + hi)
    gy = (np.arange(n_side) + 0.5) * a
    X, Y, Z = np.meshgrid(gx, gy, gy, indexing="ij")
    x = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    x = x + rng.uniform(-0.1 * a, 0.1 * a, size=x.shape)
    n = x.shape[0]
    xq = quantise(x)
    u = 1.0 + 0.5 * np.sin(2 * np.pi * xq[:, 1])
    return _pack(xq, np.full(n, 1.0 / n), u, name=f"sinusoid_{n_side}^3")


def zeldovich(n_side: int = 256, seed: int = 5, amp: float = 8.0) -> dict:
    """Lattice displaced by a Zel'dovich field: delta(k) Gaussian with
    P(k) ~ k^-2 on an n_side^3 FFT grid, psi(k) = i k delta(k) / k^2,
    x = q + amp * psi(q) / std(|psi|) * a (amp in units of the lattice
    spacing a).  m = 1/N, u = 1, v = 0.  (Shell crossing caps the density
    contrast: the 48th-neighbour distance spans only ~15x for any amp.)"""
    rng = np.random.default_rng(seed)
    n = n_side
    a = 1.0 / n
    kf = 2 * np.pi * np.fft.fftfreq(n, d=a)
    kr = 2 * np.pi * np.fft.rfftfreq(n, d=a)
    KX, KY, KZ = np.meshgrid(kf, kf, kr, indexing="ij")
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    k2[0, 0, 0] = 1.0
    white = rng.standard_normal((n, n, n))
    wk = np.fft.rfftn(white)
    delta_k = wk * np.sqrt(1.0 / k2)          # P(k) ~ k^-2  ->  |delta_k| ~ k^-1
    delta_k[0, 0, 0] = 0.0
    disp = []
    for K in (KX, KY, KZ):
        psi_k = 1j * K * delta_k / k2
        disp.append(np.fft.irfftn(psi_k, s=(n, n, n), axes=(0, 1, 2)).ravel())
    disp = np.stack(disp, axis=1)
    disp *= amp * a / np.sqrt(np.mean(np.sum(disp ** 2, axis=1)))
    g = (np.arange(n) + 0.5) * a
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    x = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1) + disp
    N = x.shape[0]
    return _pack(x, np.full(N, 1.0 / N), np.ones(N), name=f"zeldovich_{n_side}^3_amp{amp}")


def _grf(n: int, rng: np.random.Generator, slope: float = -2.0) -> np.ndarray:
    """Unit-variance Gaussian random field on an n^3 grid with P(k) ~ k^slope."""
    kf = np.fft.fftfreq(n) * n
    kr = np.fft.rfftfreq(n) * n
    KX, KY, KZ = np.meshgrid(kf, kf, kr, indexing="ij")
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    k2[0, 0, 0] = 1.0
    wk = np.fft.rfftn(rng.standard_normal((n, n, n)))
    wk *= k2 ** (slope / 4.0)
    wk[0, 0, 0] = 0.0
    g = np.fft.irfftn(wk, s=(n, n, n), axes=(0, 1, 2))
    return g / g.std()


def lognormal(n_side: int = 256, seed: int = 5, sigma: float = 4.0, grid: int | None = None) -> dict:
    """N = n_side^3 particles drawn from the density rho ~ exp(sigma G) of a
    unit-variance Gaussian field G with P(k) ~ k^-2 on a grid^3 mesh
    (grid = n_side by default): per-cell counts are one multinomial draw,
    positions uniform inside each cell.  m = 1/N, u = 1, v = 0."""
    rng = np.random.default_rng(seed)
    g = grid or n_side
    N = n_side ** 3
    G = _grf(g, rng)
    w = np.exp(sigma * (G - G.max()))
    p = (w / w.sum()).ravel()
    counts = rng.multinomial(N, p)
    cells = np.repeat(np.arange(p.size), counts)
    ix, iy, iz = np.unravel_index(cells, (g, g, g))
    x = (np.stack([ix, iy, iz], axis=1) + rng.uniform(0.0, 1.0, size=(N, 3))) / g
    return _pack(x, np.full(N, 1.0 / N), np.ones(N), name=f"lognormal_{n_side}^3_s{sigma}")


def random_box(n: int, seed: int, kind: str = "uniform", v_sigma: float = 0.0) -> dict:
    """Small random test boxes: 'uniform' i.i.d. points, 'clumped' (half in
    two Gaussian clumps of width 0.05), or 'lattice' (jittered lattice with
    n rounded down to a cube).  Masses U(0.5, 1.5)/n, energies U(0.5, 2),
    optional velocities N(0, v_sigma^2)."""
    rng = np.random.default_rng(seed)
    if kind == "lattice":
        s = int(round(n ** (1 / 3)))
        x = _jittered_lattice(s, 0.1, rng)
        n = x.shape[0]
    elif kind == "clumped":
        nu = n // 2
        c = rng.uniform(0, 1, size=(2, 3))
        w = rng.integers(0, 2, size=n - nu)
        x = np.concatenate([rng.uniform(0, 1, size=(nu, 3)),
                            c[w] + rng.normal(0, 0.05, size=(n - nu, 3))])
    else:
        x = rng.uniform(0, 1, size=(n, 3))
    m = rng.uniform(0.5, 1.5, size=n) / n
    u = rng.uniform(0.5, 2.0, size=n)
    v = rng.normal(0, v_sigma, size=(n, 3)) if v_sigma > 0 else None
    return _pack(x, m, u, v=v, name=f"random_{kind}_{n}_s{seed}")
