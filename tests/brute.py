"""O(N^2) brute-force reference used only to pin the oracle's neighbour
search: every pair's minimum-image distance is computed explicitly."""
import numpy as np


def all_pairs(x, box=1.0):
    n = x.shape[0]
    d = x[:, None, :] - x[None, :, :]
    d -= box * np.rint(d / box)
    r = np.sqrt((d * d).sum(-1))
    return d, r


def directed_sets(x, h, box=1.0):
    _, r = all_pairs(x, box)
    return r < h[:, None], r


def lattice_nngb(h_over_a, nmax=4):
    """(32/3) sum over integer vectors n of w(|n| a / h): the weighted
    neighbour number of a perfect cubic lattice, by explicit enumeration."""
    g = np.arange(-nmax, nmax + 1)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    rr = np.sqrt(X ** 2 + Y ** 2 + Z ** 2).ravel() / h_over_a
    w = np.where(rr <= 0.5, 1 - 6 * rr ** 2 + 6 * rr ** 3, np.where(rr <= 1, 2 * (1 - rr) ** 3, 0.0))
    return 32.0 / 3.0 * w.sum(), int((rr < 1).sum()), rr
