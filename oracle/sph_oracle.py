"""FP64 CPU oracle for the SPH density / smoothing-length / force path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this module.  It shares no code with the CUDA library: it does not import
the package, and the package does not import it.

What it computes (Gonnet, "Efficient and Scalable Algorithms for Smoothed
Particle Hydrodynamics on Hybrid Shared/Distributed-Memory Architectures",
Section 2.1):

* the cubic-spline kernel W(r, h) with support radius h (the piecewise
  cubic printed after Eq. (interp));
* the density rho_i = sum_{r_ij < h_i} m_j W(r_ij, h_i), Eq. (rho),
  including the self term j = i;
* the weighted neighbour number N_i = (4/3) pi h_i^3 sum_j W(r_ij, h_i),
  Eq. (nneigh), and h_i chosen so that N_i = N_ngb (48), found here as the
  exact root (bisection on a bracket, then Newton polish) rather than the
  paper's "+-1" window;
* P_i = rho_i u_i (gamma - 1) and Omega_i = 1 + h_i/(3 rho_i) d rho_i/d h_i
  (text after Eq. (dudt)), gamma = 5/3;
* dv_i/dt, Eq. (dvdt), over r_ij < max(h_i, h_j), and du_i/dt, Eq. (dudt),
  over r_ij < h_i, with grad W(r, h) = dW/dr (x_i - x_j)/r (zero at r = 0);
* the Monaghan-Balsara artificial viscosity added to Eq. (dvdt) and
  Eq. (dudt), the velocity divergence and curl it needs, the time-step
  criterion Eq. (dt) and one velocity-Verlet step (Section 4.1; readings
  beside the code);
* the reverse-mode gradient of any linear functional of (rho, dv/dt, du/dt)
  with respect to positions, masses and internal energies, with h
  differentiated implicitly through N_i(h_i, x) = N_ngb.  The paper has no
  adjoint; this is the chain rule applied to the equations above.

Neighbour search is a library primitive (scipy's cKDTree with a periodic
box) followed by the exact predicate r < h written out here.  Nothing is
blocked, fused, sorted or reordered beyond what the equations state.
Everything is float64.  Inputs m, u, v arrive as float32 values (what the
GPU receives) and are widened here.

Readings of the paper taken where it is silent or inconsistent:
  * strict r < h in Eq. (rho) (W vanishes at r = h in any case);
  * the self term j = i counts in rho, d rho/dh and N_ngb, not in forces;
  * grad_r W points along x_i - x_j, so dv_i/dt of Eq. (dvdt) is the
    acceleration of particle i (this conserves momentum exactly);
  * coincident particles (r = 0, j != i) are neighbours with zero gradient.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
from scipy.spatial import cKDTree

N_NGB = 48.0
GAMMA = 5.0 / 3.0
SIGMA = 8.0 / math.pi          # 3D normalisation of the cubic spline, W = SIGMA/h^3 w(q)
NGB_FAC = 32.0 / 3.0           # (4/3) pi h^3 * SIGMA / h^3


# --------------------------------------------------------------------------
# Kernel (Section 2.1, the piecewise cubic after Eq. (interp))
# --------------------------------------------------------------------------
def w(q):
    """Dimensionless cubic spline: 1 - 6q^2 + 6q^3 on [0, 1/2],
    2(1 - q)^3 on (1/2, 1], 0 beyond."""
    q = np.asarray(q, dtype=np.float64)
    return np.where(q <= 0.5, 1.0 - 6.0 * q * q + 6.0 * q ** 3,
                    np.where(q <= 1.0, 2.0 * (1.0 - q) ** 3, 0.0))


def dw(q):
    """dw/dq of the piecewise cubic."""
    q = np.asarray(q, dtype=np.float64)
    return np.where(q <= 0.5, -12.0 * q + 18.0 * q * q,
                    np.where(q <= 1.0, -6.0 * (1.0 - q) ** 2, 0.0))


def d2w(q):
    """d^2w/dq^2 of the piecewise cubic (continuous: the spline is C^2)."""
    q = np.asarray(q, dtype=np.float64)
    return np.where(q <= 0.5, -12.0 + 36.0 * q,
                    np.where(q <= 1.0, 12.0 * (1.0 - q), 0.0))


def W(r, h):
    """W(r, h) = 8/(pi h^3) w(r/h)."""
    return SIGMA / h ** 3 * w(r / h)


def G(r, h):
    """dW/dr = 8/(pi h^4) w'(r/h); grad_i W = G (x_i - x_j)/r."""
    return SIGMA / h ** 4 * dw(r / h)


def dW_dh(r, h):
    """dW/dh at fixed r = -8/(pi h^4) (3 w + q w')."""
    q = r / h
    return -SIGMA / h ** 4 * (3.0 * w(q) + q * dw(q))


def d2W_dh2(r, h):
    """d^2W/dh^2 at fixed r = 8/(pi h^5) (12 w + 8 q w' + q^2 w'')."""
    q = r / h
    return SIGMA / h ** 5 * (12.0 * w(q) + 8.0 * q * dw(q) + q * q * d2w(q))


def dG_dr(r, h):
    """d^2W/dr^2 = 8/(pi h^5) w''(r/h)."""
    return SIGMA / h ** 5 * d2w(r / h)


def dG_dh(r, h):
    """d^2W/(dr dh) = -8/(pi h^5) (4 w' + q w'')."""
    q = r / h
    return -SIGMA / h ** 5 * (4.0 * dw(q) + q * d2w(q))


# --------------------------------------------------------------------------
# Neighbour search (library primitive + exact predicate)
# --------------------------------------------------------------------------
def min_image(d, box):
    return d - box * np.rint(d / box)


class Neighbours:
    """Candidate pairs from a periodic cKDTree ball query (radius inflated by
    1e-9 so that the library's own rounding can never drop a pair), kept as
    flat arrays (row, j, d = x_i - x_j minimum image, r)."""

    def __init__(self, x, box=1.0):
        self.x = np.ascontiguousarray(x, dtype=np.float64)
        self.box = float(box)
        self.tree = cKDTree(self.x, boxsize=self.box)

    def query(self, idx, radius):
        idx = np.asarray(idx, dtype=np.int64)
        radius = np.broadcast_to(np.asarray(radius, dtype=np.float64), idx.shape)
        lists = self.tree.query_ball_point(self.x[idx], r=radius * (1.0 + 1e-9),
                                           workers=-1, return_sorted=False)
        counts = np.fromiter((len(l) for l in lists), dtype=np.int64, count=len(lists))
        j = np.fromiter(itertools.chain.from_iterable(lists), dtype=np.int64,
                        count=int(counts.sum()))
        row = np.repeat(np.arange(idx.size, dtype=np.int64), counts)
        d = min_image(self.x[idx[row]] - self.x[j], self.box)
        r = np.sqrt(np.einsum("ij,ij->i", d, d))
        return row, j, d, r


def _rowsum(row, vals, n):
    return np.bincount(row, weights=vals, minlength=n)


# --------------------------------------------------------------------------
# Density at given h, Eq. (rho) and Eq. (nneigh)
# --------------------------------------------------------------------------
def density_at(nb: Neighbours, m, h, idx=None):
    """rho_i, d rho_i/dh, N_i, dN_i/dh and the directed neighbour count
    (r_ij < h_i, self included) for particles ``idx`` at the given h."""
    m = np.asarray(m, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    if idx is None:
        idx = np.arange(nb.x.shape[0])
    idx = np.asarray(idx, dtype=np.int64)
    hi = h[idx]
    row, j, d, r = nb.query(idx, hi)
    keep = r < hi[row]
    row, j, r = row[keep], j[keep], r[keep]
    hr = hi[row]
    q = r / hr
    n = idx.size
    rho = _rowsum(row, m[j] * W(r, hr), n)
    drho = _rowsum(row, m[j] * dW_dh(r, hr), n)
    nngb = NGB_FAC * _rowsum(row, w(q), n)
    dnngb = NGB_FAC * _rowsum(row, -q * dw(q) / hr, n)
    count = np.bincount(row, minlength=n)
    return dict(rho=rho, drho_dh=drho, nngb=nngb, dnngb_dh=dnngb, count=count)


# --------------------------------------------------------------------------
# Smoothing length: root of N_i(h) = N_ngb (Eq. (nneigh), Newton with the
# derivative computed alongside the sums, kept inside a bisection bracket)
# --------------------------------------------------------------------------
def solve_h(nb: Neighbours, h_guess, idx=None, n_ngb=N_NGB, rtol=1e-14, max_iter=200):
    """Root of (32/3) sum_j w(r_ij/h) = n_ngb for each particle in ``idx``
    (``h_guess`` is a scalar or a full-length array).

    The bracket's upper end starts at the guess and grows by 1.5x until
    N(h_hi) >= n_ngb; every neighbour within h_hi is then a fixed candidate
    set, and the root is found by Newton steps (dN/dh summed alongside N)
    that fall back to bisection whenever they leave the bracket, until
    |dh| <= rtol h.  N(h) is continuous and non-decreasing with N(0+) = 32/3
    (the self term), so the root in (0, h_hi] is unique."""
    n_all = nb.x.shape[0]
    if idx is None:
        idx = np.arange(n_all)
    idx = np.asarray(idx, dtype=np.int64)
    hg = np.asarray(h_guess, dtype=np.float64)
    if hg.ndim == 0:
        hg = np.full(n_all, float(hg))
    n = idx.size
    h_up = hg[idx].copy()
    todo = np.arange(n)
    rows_all, r_all = [], []
    while todo.size:
        row, j, d, r = nb.query(idx[todo], h_up[todo])
        nup = NGB_FAC * _rowsum(row, w(r / h_up[todo][row]), todo.size)
        ok = nup >= n_ngb
        sel = ok[row]
        rows_all.append(todo[row[sel]])
        r_all.append(r[sel])
        h_up[todo[~ok]] *= 1.5
        todo = todo[~ok]
    row = np.concatenate(rows_all)
    r = np.concatenate(r_all)
    lo = np.zeros(n)
    hi = h_up.copy()
    h = hg[idx].copy()
    active = np.ones(n, dtype=bool)
    for _ in range(max_iter):
        if not active.any():
            break
        sel = active[row]
        rr, ro = r[sel], row[sel]
        hh = h[ro]
        q = rr / hh
        N = NGB_FAC * _rowsum(ro, w(q), n)
        dN = NGB_FAC * _rowsum(ro, -q * dw(q) / hh, n)
        f = N - n_ngb
        lo = np.where(active & (f < 0), h, lo)
        hi = np.where(active & (f >= 0), h, hi)
        with np.errstate(divide="ignore", invalid="ignore"):
            hn = h - f / dN
        bad = ~np.isfinite(hn) | (hn <= lo) | (hn >= hi) | (dN <= 0)
        hn = np.where(bad, 0.5 * (lo + hi), hn)
        conv = (np.abs(hn - h) <= rtol * h) | (f == 0)
        h = np.where(active & (f != 0), hn, h)
        active = active & ~conv
    if active.any():
        raise RuntimeError(f"oracle h-solve did not converge for {int(active.sum())} particles")
    return h


# --------------------------------------------------------------------------
# Ghost quantities (text after Eq. (dudt))
# --------------------------------------------------------------------------
def ghost(h, rho, drho_dh, u, gamma=GAMMA):
    """Omega_i = 1 + h_i/(3 rho_i) d rho_i/dh, P_i = (gamma-1) rho_i u_i and
    the force prefactor A_i = P_i / (Omega_i rho_i^2)."""
    u = np.asarray(u, dtype=np.float64)
    omega = 1.0 + h * drho_dh / (3.0 * rho)
    P = (gamma - 1.0) * rho * u
    A = P / (omega * rho * rho)
    return omega, P, A


# --------------------------------------------------------------------------
# Pair sets
# --------------------------------------------------------------------------
def directed_pairs(nb: Neighbours, h, idx=None):
    """(i, j, d, r) for r_ij < h_i, self pairs included (row indices refer
    to ``idx``; i is the particle index)."""
    if idx is None:
        idx = np.arange(nb.x.shape[0])
    idx = np.asarray(idx, dtype=np.int64)
    row, j, d, r = nb.query(idx, h[idx])
    keep = r < h[idx][row]
    return idx[row[keep]], j[keep], d[keep], r[keep]


def force_pairs_all(nb: Neighbours, h):
    """Ordered pairs (i, j), i != j, with r_ij < max(h_i, h_j) over the whole
    set: the union of the directed sets r < h_i and their transposes."""
    i, j, d, r = directed_pairs(nb, h)
    nz = i != j
    i, j = i[nz], j[nz]
    n = nb.x.shape[0]
    key = np.concatenate([i * n + j, j * n + i])
    key = np.unique(key)
    I, J = key // n, key % n
    d = min_image(nb.x[I] - nb.x[J], nb.box)
    r = np.sqrt(np.einsum("ij,ij->i", d, d))
    return I, J, d, r


class _ReverseReach:
    """Finds, for query particles, every j with r_ij < ub_j where ub_j is an
    upper bound on h_j: particles are binned by ub (factor-2 bins) and each
    bin gets its own tree, queried at the bin's largest ub."""

    def __init__(self, x, ub, box):
        self.x, self.box = x, box
        self.ub = ub
        e = np.floor(np.log2(ub)).astype(np.int64)
        self.bins = []
        for b in np.unique(e):
            members = np.nonzero(e == b)[0]
            self.bins.append((members, cKDTree(x[members], boxsize=box), float(ub[members].max())))

    def query(self, idx):
        out_i, out_j = [], []
        for members, tree, R in self.bins:
            lists = tree.query_ball_point(self.x[idx], r=R * (1 + 1e-9), workers=-1,
                                          return_sorted=False)
            counts = np.fromiter((len(l) for l in lists), dtype=np.int64, count=len(lists))
            loc = np.fromiter(itertools.chain.from_iterable(lists), dtype=np.int64,
                              count=int(counts.sum()))
            rows = np.repeat(idx, counts)
            jj = members[loc]
            d = min_image(self.x[rows] - self.x[jj], self.box)
            r = np.sqrt(np.einsum("ij,ij->i", d, d))
            keep = r < self.ub[jj] * (1 + 1e-9)
            out_i.append(rows[keep])
            out_j.append(jj[keep])
        return np.concatenate(out_i), np.concatenate(out_j)


def h_upper_bound(nb: Neighbours, k=18):
    """An upper bound on each particle's solved h: N(h) >= (32/3) w(1/2)
    * #{r < h/2} = (8/3) #{r < h/2}, so with 18 particles (self included)
    inside h/2, N(h) >= 48.  Hence h <= 2 * (distance to the 18th nearest)."""
    dist, _ = nb.tree.query(nb.x, k=k, workers=-1)
    return 2.0 * dist[:, -1] * (1 + 1e-12)


# --------------------------------------------------------------------------
# Force (Eq. (dvdt) and Eq. (dudt))
# --------------------------------------------------------------------------
def force_from_pairs(I, J, d, r, n, m, h, A, v):
    """a_i = -sum_j m_j [A_i G(r,h_i) + A_j G(r,h_j)] (x_i - x_j)/r and
    du_i/dt = A_i sum_{r<h_i} m_j (v_i - v_j).(x_i - x_j)/r G(r, h_i),
    summed over the ordered pairs (I, J); rows are I.  Pairs with r = 0
    contribute nothing (the gradient of W vanishes there)."""
    m = np.asarray(m, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    pos = r > 0
    I, J, d, r = I[pos], J[pos], d[pos], r[pos]
    xhat = d / r[:, None]
    Gi = G(r, h[I])
    Gj = G(r, h[J])
    phi = A[I] * Gi + A[J] * Gj
    c = -(m[J] * phi)[:, None] * xhat
    a = np.stack([np.bincount(I, weights=c[:, k], minlength=n) for k in range(3)], axis=1)
    vij = v[I] - v[J]
    e = A[I] * m[J] * Gi * np.einsum("ij,ij->i", vij, xhat)
    du = np.bincount(I, weights=e, minlength=n)
    return a, du


def _pairs_count(I, J, n):
    return np.bincount(I, minlength=n)


# --------------------------------------------------------------------------
# Whole-set evaluation
# --------------------------------------------------------------------------
def evaluate(x, m, u, v=None, h_guess=None, box=1.0, n_ngb=N_NGB, gamma=GAMMA, h=None):
    """Full forward pass over every particle: h (solved unless given), rho,
    d rho/dh, N_ngb, Omega, P, A, dv/dt, du/dt and pair counts."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    if v is None:
        v = np.zeros((n, 3))
    nb = Neighbours(x, box)
    if h is None:
        if h_guess is None:
            h_guess = h_upper_bound(nb)
        h = solve_h(nb, h_guess, n_ngb=n_ngb)
    h = np.asarray(h, dtype=np.float64)
    den = density_at(nb, m, h)
    omega, P, A = ghost(h, den["rho"], den["drho_dh"], u, gamma)
    I, J, d, r = force_pairs_all(nb, h)
    a, du = force_from_pairs(I, J, d, r, n, m, h, A, v)
    out = dict(h=h, omega=omega, P=P, A=A, a=a, dudt=du,
               force_count=_pairs_count(I, J, n), nb=nb)
    out.update(den)
    return out


def evaluate_sample(x, m, u, sample, v=None, box=1.0, n_ngb=N_NGB, gamma=GAMMA):
    """Forward values for the particles in ``sample`` only, computed from
    scratch: h, rho, Omega of the sample and of every particle whose force
    pair set reaches it, then dv/dt and du/dt of the sample."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    if v is None:
        v = np.zeros((n, 3))
    sample = np.asarray(sample, dtype=np.int64)
    nb = Neighbours(x, box)
    ub = h_upper_bound(nb)
    h = np.full(n, np.nan)
    h[sample] = solve_h(nb, ub, idx=sample, n_ngb=n_ngb)
    # partners: j with r < h_i (i in sample) or r < h_j
    i1, j1, _, _ = directed_pairs(nb, np.where(np.isnan(h), 0.0, h), idx=sample)
    i2, j2 = _ReverseReach(x, ub, box).query(sample)
    partners = np.setdiff1d(np.unique(np.concatenate([j1, j2])), sample)
    if partners.size:
        h[partners] = solve_h(nb, ub, idx=partners, n_ngb=n_ngb)
    need = np.concatenate([sample, partners])
    den = density_at(nb, m, h, idx=need)
    rho = np.full(n, np.nan); drho = np.full(n, np.nan)
    rho[need] = den["rho"]; drho[need] = den["drho_dh"]
    omega, P, A = ghost(h, rho, drho, u, gamma)
    # exact pair set of the sample
    I = np.concatenate([i1, i2]); J = np.concatenate([j1, j2])
    key = np.unique(I * n + J)
    I, J = key // n, key % n
    d = min_image(x[I] - x[J], box)
    r = np.sqrt(np.einsum("ij,ij->i", d, d))
    keep = (I != J) & ((r < h[I]) | (r < h[J]))
    I, J, d, r = I[keep], J[keep], d[keep], r[keep]
    a, du = force_from_pairs(I, J, d, r, n, m, np.where(np.isnan(h), 1.0, h),
                             np.where(np.isnan(A), 0.0, A), v)
    res = dict(idx=sample, h=h[sample], rho=rho[sample], drho_dh=drho[sample],
               omega=omega[sample], A=A[sample], a=a[sample], dudt=du[sample],
               force_count=np.bincount(np.searchsorted(sample, I[np.isin(I, sample)]),
                                       minlength=sample.size) if np.all(np.diff(sample) > 0) else None)
    sub = density_at(nb, m, h, idx=sample)
    res["nngb"] = sub["nngb"]
    res["count"] = sub["count"]
    return res


# --------------------------------------------------------------------------
# Reverse mode (chain rule through Eq. (dvdt), (dudt), the ghost step,
# Eq. (rho) and the implicit h of Eq. (nneigh))
# --------------------------------------------------------------------------
def gradient(fwd, x, m, u, v, g_rho, g_a, g_dudt=None, gamma=GAMMA):
    """Gradient of L = sum_i g_rho_i rho_i + g_a_i . a_i + g_dudt_i du_i/dt
    with respect to x (N x 3), m and u, given a forward state from
    ``evaluate``.  Returns dict(g_x, g_m, g_u)."""
    x = np.asarray(x, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    v = np.zeros_like(x) if v is None else np.asarray(v, dtype=np.float64)
    n = x.shape[0]
    nb = fwd["nb"]
    h, rho, drho, omega, A = fwd["h"], fwd["rho"], fwd["drho_dh"], fwd["omega"], fwd["A"]
    g_rho = np.asarray(g_rho, dtype=np.float64).copy()
    g_a = np.asarray(g_a, dtype=np.float64)
    g_du = np.zeros(n) if g_dudt is None else np.asarray(g_dudt, dtype=np.float64)

    gx = np.zeros((n, 3)); gm = np.zeros(n); gA = np.zeros(n); gh = np.zeros(n)

    def scat(idx, vals, out):
        out += np.bincount(idx, weights=vals, minlength=n)

    # ---- force, Eq. (dvdt) and (dudt): ordered pairs, the i-equation terms
    I, J, d, r = force_pairs_all(nb, h)
    pos = r > 0
    I, J, d, r = I[pos], J[pos], d[pos], r[pos]
    xh = d / r[:, None]
    hi, hj = h[I], h[J]
    Gi, Gj = G(r, hi), G(r, hj)
    Gpi, Gpj = dG_dr(r, hi), dG_dr(r, hj)
    Ghi, Ghj = dG_dh(r, hi), dG_dh(r, hj)
    phi = A[I] * Gi + A[J] * Gj
    dphi = A[I] * Gpi + A[J] * Gpj
    ga_i = g_a[I]
    s = np.einsum("ij,ij->i", ga_i, xh)
    scat(I, -m[J] * Gi * s, gA)
    scat(J, -m[J] * Gj * s, gA)
    scat(J, -phi * s, gm)
    scat(I, -m[J] * A[I] * Ghi * s, gh)
    scat(J, -m[J] * A[J] * Ghj * s, gh)
    dd = -(m[J])[:, None] * (dphi[:, None] * s[:, None] * xh
                             + (phi / r)[:, None] * (ga_i - s[:, None] * xh))
    # du/dt term (only r < h_i contributes through G_i)
    vij = v[I] - v[J]
    t = np.einsum("ij,ij->i", vij, xh)
    gdu_i = g_du[I]
    scat(I, gdu_i * m[J] * Gi * t, gA)
    scat(J, gdu_i * A[I] * Gi * t, gm)
    scat(I, gdu_i * A[I] * m[J] * Ghi * t, gh)
    dd = dd + (gdu_i * A[I] * m[J])[:, None] * (Gpi[:, None] * t[:, None] * xh
                                               + (Gi / r)[:, None] * (vij - t[:, None] * xh))
    for k in range(3):
        scat(I, dd[:, k], gx[:, k])
        scat(J, -dd[:, k], gx[:, k])

    # ---- ghost: A = (gamma-1) u / (Omega rho), Omega = 1 + h rho'/(3 rho)
    gu = gA * (gamma - 1.0) / (omega * rho)
    gO = -gA * A / omega
    g_rho += -gA * A / rho
    g_rho += -gO * h * drho / (3.0 * rho * rho)
    g_drho = gO * h / (3.0 * rho)
    gh += gO * drho / (3.0 * rho)

    # ---- density, Eq. (rho), and rho' = sum m_j dW/dh: directed pairs r < h_i
    i, j, dv, rv = directed_pairs(nb, h)
    hh = h[i]
    Wv = W(rv, hh)
    Wh = dW_dh(rv, hh)
    scat(j, g_rho[i] * Wv + g_drho[i] * Wh, gm)
    scat(i, g_rho[i] * m[j] * Wh + g_drho[i] * m[j] * d2W_dh2(rv, hh), gh)
    nz = rv > 0
    i2, j2, d2, r2, h2 = i[nz], j[nz], dv[nz], rv[nz], hh[nz]
    xh2 = d2 / r2[:, None]
    coef = m[j2] * (g_rho[i2] * G(r2, h2) + g_drho[i2] * dG_dh(r2, h2))
    # ---- implicit h: lambda_i = g_h_i / (dN_i/dh_i); N_i depends on x only
    dN = NGB_FAC * np.bincount(i, weights=-(rv / hh) * dw(rv / hh) / hh, minlength=n)
    lam = gh / dN
    coef = coef - lam[i2] * NGB_FAC * dw(r2 / h2) / h2
    for k in range(3):
        scat(i2, coef * xh2[:, k], gx[:, k])
        scat(j2, -coef * xh2[:, k], gx[:, k])
    return dict(g_x=gx, g_m=gm, g_u=gu, g_h_explicit=gh, lam=lam)


# --------------------------------------------------------------------------
# FP32 neighbour predicate, reproduced exactly (pair-set parity)
# --------------------------------------------------------------------------
def _rn32(v):
    """Round float64 values that are exact integers below 2^53 to the
    nearest float32 (ties to even): one correct rounding."""
    return np.asarray(v, dtype=np.float64).astype(np.float32).astype(np.float64)


def fp32_r2_units(dk):
    """r^2 in units of 2^-48 as the FP32 expression
    fma(dz, dz, fma(dy, dy, dx*dx)) evaluates it, for integer coordinate
    differences dk (units of 2^-24, |dk| < 2^24).  Every intermediate is an
    integer below 2^53, so float64 holds it exactly and each float32
    rounding is a single correct rounding, as in the hardware FMA."""
    dk = np.asarray(dk, dtype=np.int64)
    kx, ky, kz = dk[:, 0], dk[:, 1], dk[:, 2]
    p1 = _rn32((kx * kx).astype(np.float64))
    p2 = _rn32((ky * ky).astype(np.float64) + p1)
    return _rn32((kz * kz).astype(np.float64) + p2)


def fp32_h2_units(h32):
    """fl32(h*h) for float32 h, in units of 2^-48."""
    h = np.asarray(h32, dtype=np.float32).astype(np.float64)
    return _rn32(h * h) * 2.0 ** 48


def pairs_fp32(x, h32, phase="density", box=1.0):
    """Exact pair sets of the FP32 predicate on positions quantised to
    multiples of 2^-24 in a unit box: phase 'density' gives (i, j) with
    fl32 r^2 < fl32 h_i^2 (self included); phase 'force' gives i != j with
    fl32 r^2 < max(fl32 h_i^2, fl32 h_j^2).  Returned as sorted int64 keys
    i * N + j."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    h32 = np.asarray(h32, dtype=np.float32)
    hq = h32.astype(np.float64) * (1 + 1e-5)
    nb = Neighbours(x, box)
    k = np.rint(x * 2.0 ** 24).astype(np.int64)
    if phase == "density":
        row, j, _, _ = nb.query(np.arange(n), hq)
        I = row
    else:
        i1, j1, _, _ = nb.query(np.arange(n), hq)
        I = np.concatenate([i1, j1]); j = np.concatenate([j1, i1])
    dk = k[I] - k[j]
    dk = dk - (2 ** 24) * np.rint(dk / 2.0 ** 24).astype(np.int64)
    r2 = fp32_r2_units(dk)
    h2 = fp32_h2_units(h32)
    if phase == "density":
        keep = r2 < h2[I]
    else:
        keep = (I != j) & ((r2 < h2[I]) | (r2 < h2[j]))
    return np.unique(I[keep] * n + j[keep])


# --------------------------------------------------------------------------
# Artificial viscosity and the time-step criterion (Section 4.1: the
# Monaghan-Balsara terms added to Eq. (dvdt) and Eq. (dudt), and Eq. (dt)).
# Readings where the printed formulas are garbled or silent:
#   * the switch is Balsara's, f_i = |div v_i| / (|div v_i| + |curl v_i|
#     + 1e-4 c_i/h_i): the printed numerator |curl v_i| would switch the
#     viscosity on in pure shear and off in pure compression, the opposite
#     of its stated purpose, and the printed c_j/h_j has no j in scope;
#   * c_i = sqrt(gamma (gamma - 1) u_i), the ideal-gas sound speed;
#   * the viscous sums run over the pressure force's pair set,
#     r_ij < max(h_i, h_j) (the printed h-hat_ij);
#   * div v_i and curl v_i sum over the density loop's set r_ij < h_i (the
#     self term contributes nothing: v_i - v_i = 0);
#   * the maximum in Eq. (dt) runs over the same force pairs; a particle
#     with none takes c_i + c_i.
# --------------------------------------------------------------------------
def sound_speed(u, gamma=GAMMA):
    """c_i = sqrt(gamma (gamma - 1) u_i)."""
    return np.sqrt(gamma * (gamma - 1.0) * np.asarray(u, dtype=np.float64))


def velocity_derivatives(nb: Neighbours, m, v, h, rho):
    """div v_i = (1/rho_i) sum_j m_j (v_j - v_i) . grad W(r_ij, h_i) and
    curl v_i = -(1/rho_i) sum_j m_j (v_j - v_i) x grad W(r_ij, h_i) over
    r_ij < h_i, with grad W = G(r, h) (x_i - x_j)/r (Section 4.1)."""
    n = nb.x.shape[0]
    m = np.asarray(m, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    i, j, d, r = directed_pairs(nb, h)
    pos = r > 0
    i, j, d, r = i[pos], j[pos], d[pos], r[pos]
    gw = (G(r, h[i]) / r)[:, None] * d                   # grad_i W(r_ij, h_i)
    dv = v[j] - v[i]
    div = np.bincount(i, weights=m[j] * np.einsum("ij,ij->i", dv, gw), minlength=n) / rho
    cr = np.cross(dv, gw) * m[j][:, None]
    curl = -np.stack([np.bincount(i, weights=cr[:, k], minlength=n) for k in range(3)],
                     axis=1) / rho[:, None]
    return div, curl


def balsara(div, curl, c, h):
    """f_i = |div v_i| / (|div v_i| + |curl v_i| + 1e-4 c_i/h_i)."""
    ad = np.abs(div)
    ac = np.linalg.norm(curl, axis=1)
    return ad / (ad + ac + 1e-4 * c / h)


def viscosity_from_pairs(I, J, d, r, n, m, v, h, rho, c, f, alpha):
    """The viscous terms over the ordered force pairs (I, J), rows I:
    dv_i/dt += -(1/4) sum_j m_j Pi_ij (grad W(r,h_i) + grad W(r,h_j)) (f_i + f_j),
    du_i/dt += (1/8) sum_j m_j Pi_ij v_ij . (grad W(r,h_i) + grad W(r,h_j)) (f_i + f_j),
    Pi_ij = -alpha (c_i + c_j - 3 w_ij) w_ij / (rho_i + rho_j),
    w_ij = min(0, v_ij . r_ij / r_ij), v_ij = v_i - v_j (Section 4.1)."""
    m = np.asarray(m, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    pos = r > 0
    I, J, d, r = I[pos], J[pos], d[pos], r[pos]
    xhat = d / r[:, None]
    vij = v[I] - v[J]
    wij = np.minimum(0.0, np.einsum("ij,ij->i", vij, xhat))
    Pi = -alpha * (c[I] + c[J] - 3.0 * wij) * wij / (rho[I] + rho[J])
    gsum = (G(r, h[I]) + G(r, h[J]))[:, None] * xhat     # grad W_i + grad W_j
    fs = f[I] + f[J]
    ca = -0.25 * (m[J] * Pi * fs)[:, None] * gsum
    a = np.stack([np.bincount(I, weights=ca[:, k], minlength=n) for k in range(3)], axis=1)
    e = 0.125 * m[J] * Pi * fs * np.einsum("ij,ij->i", vij, gsum)
    du = np.bincount(I, weights=e, minlength=n)
    return a, du


def cfl_dt(I, J, d, r, n, v, h, c, c_cfl):
    """Eq. (dt): dt_i = C_CFL 2 h_i / max_j (c_i + c_j + max(0, -3 r_ij . v_ij / r_ij))
    over the force pairs (I, J); c_i + c_i for a particle without any."""
    v = np.asarray(v, dtype=np.float64)
    sig = 2.0 * c.copy()
    pos = r > 0
    I, J, d, r = I[pos], J[pos], d[pos], r[pos]
    rv = np.einsum("ij,ij->i", d, v[I] - v[J]) / r
    s = c[I] + c[J] + np.maximum(0.0, -3.0 * rv)
    vmax = np.full(n, -np.inf)
    np.maximum.at(vmax, I, s)
    has = np.isfinite(vmax)
    sig[has] = vmax[has]
    return c_cfl * 2.0 * h / sig


def evaluate_viscosity(fwd, x, m, u, v, alpha=0.8, c_cfl=0.25, gamma=GAMMA):
    """Viscous accelerations and heating, the Balsara switch, div/curl v and
    the time steps at the solved h of ``fwd`` (an ``evaluate`` result).
    alpha = 0.8 and C_CFL = 1/4 are the values of the paper's runs."""
    nb = fwd["nb"]
    n = nb.x.shape[0]
    h, rho = fwd["h"], fwd["rho"]
    c = sound_speed(u, gamma)
    div, curl = velocity_derivatives(nb, m, v, h, rho)
    f = balsara(div, curl, c, h)
    I, J, d, r = force_pairs_all(nb, h)
    a, du = viscosity_from_pairs(I, J, d, r, n, m, v, h, rho, c, f, alpha)
    dt = cfl_dt(I, J, d, r, n, v, h, c, c_cfl)
    return dict(a_visc=a, dudt_visc=du, div=div, curl=curl, balsara=f, c=c, dt=dt)


# --------------------------------------------------------------------------
# Time integration (Section 4.1: velocity Verlet).  Readings: the
# kick-drift-kick form with one global step (the multiple time-stepping of
# Section 4.1 is a scheduling device); because du/dt and the viscosity
# depend on the velocities, the closing kick uses forces evaluated with the
# velocities and energies predicted to the end of the step, v + dt a(t) and
# u + dt du/dt(t), and every step starts from forces evaluated at its actual
# state (reusing the predicted-state forces would break the step's exact
# energy bookkeeping); h is solved afresh at every evaluation, from the
# previous h.  The total energy error of a step is then dt^2/8 sum_i m_i
# |a_i(t + dt) - a_i(t)|^2 >= 0 for inviscid flow: third order over a run.
# --------------------------------------------------------------------------
def accelerations(x, m, u, v, h_guess, alpha=0.8, box=1.0, gamma=GAMMA):
    """dv/dt and du/dt with the viscous terms (alpha > 0) at one state."""
    fwd = evaluate(x, m, u, v=v, h_guess=h_guess, box=box, gamma=gamma)
    a, du = fwd["a"], fwd["dudt"]
    if alpha > 0:
        vis = evaluate_viscosity(fwd, x, m, u, v, alpha, 0.25, gamma)
        a, du = a + vis["a_visc"], du + vis["dudt_visc"]
    return a, du, fwd


def verlet_step(x, v, u, m, dt, h_guess, alpha=0.8, box=1.0, gamma=GAMMA):
    """One velocity-Verlet (kick-drift-kick) step of the SPH equations.
    Returns x, v, u at t + dt and the h solved there."""
    x = np.asarray(x, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    a0, du0, f0 = accelerations(x, m, u, v, h_guess, alpha, box, gamma)
    h_guess = f0["h"]
    vh = v + 0.5 * dt * a0
    uh = u + 0.5 * dt * du0
    x1 = np.mod(x + dt * vh, box)
    a1, du1, f1 = accelerations(x1, m, uh + 0.5 * dt * du0, vh + 0.5 * dt * a0, h_guess, alpha, box,
                                gamma)
    return x1, vh + 0.5 * dt * a1, uh + 0.5 * dt * du1, f1["h"]
