"""The oracle's own FP64 discrete Fourier transform (test-only).

Definition: X[k] = sum_j x[j] exp(sign * 2 pi i j k / n) along one axis;
sign = -1 is the forward transform used for delta(k) in Sec. 2.1
(eq. delta_pi_k), sign = +1 the unnormalised inverse.

Lengths up to 64 are evaluated as a direct matrix product with the DFT
matrix. Longer (composite) lengths use one textbook Cooley-Tukey split
n = n1 * n2, j = n2*j1 + j2, k = k1 + n1*k2:

    X[k1 + n1 k2] = sum_j2 W_n^(j2 k1) [sum_j1 x[n2 j1 + j2] W_n1^(j1 k1)] W_n2^(j2 k2)

with W_m = exp(sign * 2 pi i / m), applied recursively. Angles are reduced
modulo n in integers before cos/sin so that twiddles are accurate to FP64.
"""
from __future__ import annotations

import numpy as np

_DIRECT_MAX = 64


def _roots(idx: np.ndarray, n: int, sign: int) -> np.ndarray:
    m = np.mod(idx, n).astype(np.float64)
    ang = 2.0 * np.pi * m / n
    return np.cos(ang) + 1j * sign * np.sin(ang)


def dft_matrix(n: int, sign: int) -> np.ndarray:
    j = np.arange(n)
    return _roots(np.outer(j, j), n, sign)


def _split(n: int):
    n1 = 1
    while n1 * n1 < n:
        n1 *= 2
    if n % n1:
        return None
    return n1, n // n1


def dft_last(x: np.ndarray, sign: int) -> np.ndarray:
    """DFT along the last axis of a complex array."""
    n = x.shape[-1]
    if n <= _DIRECT_MAX or _split(n) is None:
        return x @ dft_matrix(n, sign).T
    n1, n2 = _split(n)
    lead = x.shape[:-1]
    y = x.reshape(lead + (n1, n2))                   # [.., j1, j2]
    y = np.swapaxes(y, -1, -2)                       # [.., j2, j1]
    y = dft_last(y, sign)                            # [.., j2, k1]
    j2 = np.arange(n2)[:, None]
    k1 = np.arange(n1)[None, :]
    y = y * _roots(j2 * k1, n, sign)                 # twiddle W_n^(j2 k1)
    y = np.swapaxes(y, -1, -2)                       # [.., k1, j2]
    y = dft_last(y, sign)                            # [.., k1, k2]
    y = np.swapaxes(y, -1, -2)                       # [.., k2, k1] -> k1 + n1 k2
    return y.reshape(lead + (n,))


def dft_axis(x: np.ndarray, axis: int, sign: int) -> np.ndarray:
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    return np.moveaxis(dft_last(np.ascontiguousarray(x), sign), -1, axis)


def dft3(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalised 3D DFT over all three axes."""
    y = np.asarray(x, dtype=np.complex128)
    for ax in (2, 1, 0):
        y = dft_axis(y, ax, sign)
    return y
