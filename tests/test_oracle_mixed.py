"""Pins of the reduced-precision arithmetic model (oracle/mixed.py).

The model rounds to bfloat16 by the IEEE rule (nearest, ties to even) and
keeps three of the four products of a hi + lo split.  Pinned by: known
roundings at and around ties; the reconstruction bound of the split; exact
products on bfloat16-representable inputs; the split-product bound against
exact dot products (and that one bfloat16 product per term would miss it by
orders of magnitude, so the bound is not vacuous); the split DFT of a line
against numpy's FFT.
"""

import numpy as np
import pytest

from oracle import mixed as X


def test_bf16_rounding_at_and_around_ties():
    one = np.float32(1.0)
    # spacing of bfloat16 at 1 is 2^-7; 1 + 2^-8 is a tie -> even (1)
    assert X.bf16(one + np.float32(2.0 ** -8)) == 1.0
    # 1 + 3 * 2^-8 is a tie between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
    assert X.bf16(np.float32(1.0 + 3 * 2.0 ** -8)) == np.float32(1.0 + 2.0 ** -6)
    # just above a tie rounds up, just below rounds down
    assert X.bf16(np.float32(1.0 + 2.0 ** -8 + 2.0 ** -20)) == np.float32(1.0 + 2.0 ** -7)
    assert X.bf16(np.float32(1.0 + 2.0 ** -8 - 2.0 ** -20)) == 1.0
    # sign symmetry and representable values unchanged
    assert X.bf16(np.float32(-(1.0 + 3 * 2.0 ** -8))) == np.float32(-(1.0 + 2.0 ** -6))
    for v in (0.0, 3.0, -0.15625, 2.0 ** 100, 2.0 ** -100, 1.0 + 2.0 ** -7):
        assert X.bf16(np.float32(v)) == np.float32(v)
    # FP32's exponent range: no overflow at 1e38
    assert np.isfinite(X.bf16(np.float32(1e38)))


def test_split_reconstructs_within_two_roundings():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-40, 40, 20000))).astype(np.float32)
    hi, lo = X.split(x)
    assert np.array_equal(X.bf16(hi), hi) and np.array_equal(X.bf16(lo), lo)
    xd = x.astype(np.float64)
    assert np.all(np.abs(xd - hi) <= 2.0 ** -8 * np.abs(xd))
    assert np.all(np.abs(xd - hi - lo) <= 2.0 ** -16 * np.abs(xd))


def test_split_dot_is_exact_on_bfloat16_inputs():
    rng = np.random.default_rng(1)
    a = X.bf16(rng.standard_normal((50, 64)))
    b = X.bf16(rng.standard_normal((50, 64)))
    exact = np.sum(a.astype(np.float64) * b.astype(np.float64), axis=1)
    assert np.array_equal(X.split_dot(a, b), exact)


@pytest.mark.parametrize("K", [16, 512, 1080])
def test_split_dot_error_bound(K):
    rng = np.random.default_rng(K)
    a = rng.standard_normal((400, K)).astype(np.float32)
    b = rng.uniform(-1, 1, (400, K)).astype(np.float32)
    exact = np.sum(a.astype(np.float64) * b.astype(np.float64), axis=1)
    mag = np.sum(np.abs(a.astype(np.float64) * b), axis=1)
    err = np.abs(X.split_dot(a, b) - exact) / mag
    assert err.max() <= X.SPLIT_BOUND
    # typical size: about 2^-16 of the terms, or less
    assert np.sqrt(np.mean(err ** 2)) < 2.0 ** -16
    # one bfloat16 product per term is ~2^-9 of the terms / sqrt(K) typical:
    # orders of magnitude above the split
    plain = np.abs(X.plain_bf16_dot(a, b) - exact) / mag
    assert np.sqrt(np.mean(plain ** 2)) > 64 * np.sqrt(np.mean(err ** 2))


@pytest.mark.parametrize("sign", [-1, 1])
def test_split_dft_matches_fft(sign):
    rng = np.random.default_rng(5 + sign)
    Q, K = 540, 256
    x = rng.standard_normal(K) + 1j * rng.standard_normal(K)
    got = X.dft_split(x, Q, sign)
    xp = np.zeros(Q, complex)
    xp[:K] = x
    ref = np.fft.fft(xp) if sign < 0 else np.fft.ifft(xp) * Q
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    # within a few 2^-16 (the split products), but visibly rounded
    assert 2.0 ** -24 < rel < 4 * 2.0 ** -16
