"""Pins of the oracle's exact reproduction of the FP32 neighbour predicate
fma(dz, dz, fma(dy, dy, dx*dx)) < fl32(h*h): an independent emulation in
exact rational arithmetic (round to nearest, ties to even, 24-bit
significand) must agree on every pair."""
from fractions import Fraction

import numpy as np

from oracle import sph_oracle as O
import synth.configs as C
from tests.brute import all_pairs


def rn32(v: Fraction) -> Fraction:
    if v == 0:
        return v
    assert v > 0
    e = v.numerator.bit_length() - v.denominator.bit_length()
    if Fraction(2) ** e > v:
        e -= 1
    scale = Fraction(2) ** (23 - e)          # v * scale in [2^23, 2^24)
    s = v * scale
    fl = s.numerator // s.denominator
    rem = s - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return Fraction(fl) / scale


def r2_exact(kx, ky, kz):
    p1 = rn32(Fraction(kx * kx))
    p2 = rn32(Fraction(ky * ky) + p1)
    return rn32(Fraction(kz * kz) + p2)


def test_r2_emulation_matches_rational_rounding():
    rng = np.random.default_rng(0)
    k = rng.integers(-(1 << 22), 1 << 22, size=(3000, 3))
    k[:1000] >>= rng.integers(0, 20, size=(1000, 1))   # many magnitudes
    got = O.fp32_r2_units(k)
    for row, g in zip(k, got):
        assert Fraction(g) == r2_exact(*map(int, row))


def test_h2_emulation_matches_rational_rounding():
    rng = np.random.default_rng(1)
    h = rng.uniform(1e-4, 0.3, size=2000).astype(np.float32)
    got = O.fp32_h2_units(h)
    for hv, g in zip(h, got):
        hf = Fraction(float(hv))
        assert Fraction(g) == rn32(hf * hf) * 2 ** 48


def test_pair_sets_match_exact_predicate():
    d = C.random_box(300, 5, "clumped")
    x = d["x"]
    n = x.shape[0]
    h32 = np.full(n, 0.12, np.float32) * np.random.default_rng(2).uniform(0.5, 1.5, n).astype(np.float32)
    k = np.rint(x * 2 ** 24).astype(np.int64)
    dk = k[:, None, :] - k[None, :, :]
    dk -= (1 << 24) * np.rint(dk / 2.0 ** 24).astype(np.int64)
    r2 = O.fp32_r2_units(dk.reshape(-1, 3)).reshape(n, n)
    h2 = O.fp32_h2_units(h32)
    S = r2 < h2[:, None]
    got = O.pairs_fp32(x, h32, "density")
    want = np.nonzero(S.ravel())[0]
    assert np.array_equal(got, want)
    F = (r2 < h2[:, None]) | (r2 < h2[None, :])
    np.fill_diagonal(F, False)
    assert np.array_equal(O.pairs_fp32(x, h32, "force"), np.nonzero(F.ravel())[0])
    # and the FP32 sets agree with the FP64 predicate except within rounding of |r - h|
    _, r = all_pairs(x)
    diff = S != (r < h32.astype(np.float64)[:, None])
    assert np.all(np.abs(r[diff] - h32.astype(np.float64)[np.nonzero(diff)[0]]) < 1e-6)
