"""Arithmetic of the reduced-precision form, written out (TEST INFRASTRUCTURE ONLY).

The reduced-precision form evaluates the y transforms of the convolutions of
Sec. III.A as products of complex DFT matrices with the data, on bfloat16
operands split into a high and a low part, with the products accumulated in
FP32.  This module states that arithmetic in plain numpy so that the error of
a split-operand dot product can be pinned against the exact product
(tests/test_oracle_mixed.py), with no GPU code involved.

bf16(x)        x (as float32) rounded to bfloat16: 8 significant bits, FP32's
               exponent range, round to nearest with ties to even
split(x)       hi = bf16(x), lo = bf16(x - hi); x - hi is exact in float32
split_dot      sum_k hi_a hi_b + hi_a lo_b + lo_a hi_b (lo_a lo_b dropped),
               every product exact, the sum in float64
SPLIT_BOUND    a rigorous bound of the products' error: with |x - hi| <= 2^-8 |x|
               and |x - hi - lo| <= 2^-16 |x| the dropped terms are
               e_b (hi_a + lo_a) + e_a (hi_b + lo_b) + lo_a lo_b + e_a e_b,
               so |a.b - split_dot(a, b)| <= ~3 * 2^-16 * sum_k |a_k| |b_k|
dft_split      the complex DFT of one line through its real-form matrix with
               split operands (the matrix entries rounded from float64)
"""

import numpy as np

SPLIT_BOUND = 3.0 * 2.0 ** -16 * (1.0 + 2.0 ** -6)


def bf16(x):
    """x rounded to bfloat16, returned as float32: the top 16 bits of the
    float32 pattern, the dropped 16 bits rounded to nearest, ties to even."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.reshape(-1).view(np.uint32).astype(np.uint64)
    keep_lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = (u + np.uint64(0x7FFF) + keep_lsb) & np.uint64(0xFFFF0000)
    return r.astype(np.uint32).view(np.float32).reshape(f.shape)


def split(x):
    """(hi, lo) of x taken as float32."""
    f = np.asarray(x, dtype=np.float32)
    hi = bf16(f)
    lo = bf16(f - hi)
    return hi, lo


def split_dot(a, b, axis=-1):
    """Split-operand dot product of a and b along `axis` (float64 result)."""
    ah, al = (v.astype(np.float64) for v in split(a))
    bh, bl = (v.astype(np.float64) for v in split(b))
    return np.sum(ah * bh + ah * bl + al * bh, axis=axis)


def plain_bf16_dot(a, b, axis=-1):
    """One bfloat16 product per term (no split), for comparison."""
    return np.sum(bf16(a).astype(np.float64) * bf16(b).astype(np.float64), axis=axis)


def dft_split(x, Q, sign):
    """sum_k x_k exp(sign 2 pi i n k / Q), n < Q, for a complex line x of
    length K <= Q (zero beyond K), in real form with split operands:
        Re y_n = sum_k Re x_k c_nk - Im x_k s_nk
        Im y_n = sum_k Re x_k s_nk + Im x_k c_nk
    where c, s are the cosine and sine of the phase (rounded to float32, then
    split like the data)."""
    x = np.asarray(x, dtype=np.complex128)
    K = x.shape[-1]
    n = np.arange(Q)[:, None]
    k = np.arange(K)[None, :]
    phase = sign * 2.0 * np.pi * ((n * k) % Q) / Q
    c, s = np.cos(phase), np.sin(phase)
    # re_n = sum_k re_k c - im_k s;  im_n = sum_k re_k s + im_k c
    xr = x.real.astype(np.float32)
    xi = x.imag.astype(np.float32)
    A = np.concatenate([xr, xi])[None, :]                      # [1, 2K]
    Bre = np.concatenate([c, -s], axis=1).astype(np.float32)    # [Q, 2K]
    Bim = np.concatenate([s, c], axis=1).astype(np.float32)
    re = split_dot(np.broadcast_to(A, Bre.shape), Bre)
    im = split_dot(np.broadcast_to(A, Bim.shape), Bim)
    return re + 1j * im
