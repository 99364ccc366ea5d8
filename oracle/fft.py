"""Oracle: the discrete Fourier transform, written out.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The march of Eq. fov10 takes F and F^-1 along the transverse coordinate at
every step (Section 2: the FFT is what makes the method fast).  The oracle
computes them here, with no library FFT:

* ``dft``: the definition X[k] = sum_j x[j] exp(-2 pi i j k / N), as a
  matrix product with the N x N matrix of exponentials (each exponent's
  j*k reduced mod N first, so every entry is a correctly rounded root of
  unity).  Used for every length N <= 256.
* ``fft``: radix-2 decimation in time for longer transforms.  The
  sequence is cut into 16-point subsequences of stride N/16, each
  transformed by the definition; then log2(N/16) doubling stages merge
  pairs of stride-r subsequences (the even- and odd-indexed halves of a
  stride-r/2 subsequence) with X[k] = E[k] + W^k O[k],
  X[k + m] = E[k] - W^k O[k], W = exp(-2 pi i / (2m)).
* ``ifft``: x[j] = (1/N) sum_k X[k] exp(+2 pi i j k / N), taken as
  conj(fft(conj(X))) / N.

Sign convention: numpy's (forward kernel exp(-2 pi i j k / N)); the band
pairing of the propagators follows from it (see ``bpm``).  All transforms
act on the last axis and keep the leading axes as a batch.
"""

from __future__ import annotations

import functools
import math

import numpy as np

DFT_MAX = 256      # lengths up to this use the O(N^2) definition
_LEAF = 16         # leaf length of the radix-2 recursion


@functools.lru_cache(maxsize=None)
def _roots(n: int, sign: float) -> np.ndarray:
    """exp(sign * 2 pi i t / n) for t = 0..n-1, each rounded from FP64."""
    t = np.arange(n, dtype=np.float64)
    return np.exp(sign * 2j * math.pi * t / n)


@functools.lru_cache(maxsize=None)
def dft_matrix(n: int) -> np.ndarray:
    """M[k][j] = exp(-2 pi i (j k mod n) / n)."""
    j = np.arange(n)
    return _roots(n, -1.0)[np.outer(j, j) % n]


def dft(x: np.ndarray) -> np.ndarray:
    """The DFT by its definition, O(N^2), along the last axis."""
    x = np.asarray(x, dtype=np.complex128)
    return x @ dft_matrix(x.shape[-1]).T


def is_pow2(n: int) -> bool:
    return n >= 1 and (n & (n - 1)) == 0


def fft(x: np.ndarray) -> np.ndarray:
    """Forward DFT along the last axis (definition for N <= 256, radix-2
    decimation in time above; N must then be a power of two)."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    if n <= DFT_MAX:
        return dft(x)
    if not is_pow2(n):
        raise ValueError(f"radix-2 FFT needs a power-of-two length, got {n}")
    lead = x.shape[:-1]
    m = _LEAF
    r = n // m
    # y[..., s, k] = DFT_m of the stride-r subsequence x[s], x[s + r], ...
    sub = np.swapaxes(x.reshape(lead + (m, r)), -1, -2)
    y = sub @ dft_matrix(m).T
    while r > 1:
        half = r // 2
        even = y[..., :half, :]            # subsequence s: even elements at stride r/2
        odd = y[..., half:, :]             # subsequence s + r/2: odd elements
        wo = _roots(2 * m, -1.0)[:m] * odd
        y = np.concatenate([even + wo, even - wo], axis=-1)
        m *= 2
        r = half
    return y[..., 0, :]


def ifft(spec: np.ndarray) -> np.ndarray:
    """Inverse DFT along the last axis, with the 1/N factor."""
    spec = np.asarray(spec, dtype=np.complex128)
    return np.conj(fft(np.conj(spec))) / spec.shape[-1]


def fft2(x: np.ndarray) -> np.ndarray:
    """2D DFT over the last two axes (one axis after the other)."""
    y = fft(x)
    return np.swapaxes(fft(np.swapaxes(y, -1, -2)), -1, -2)


def ifft2(spec: np.ndarray) -> np.ndarray:
    y = ifft(spec)
    return np.swapaxes(ifft(np.swapaxes(y, -1, -2)), -1, -2)


def fftfreq(n: int, d: float) -> np.ndarray:
    """Frequencies of the DFT bins in cycles per unit of d: the signed bin
    index (m for m < n/2, m - n from m = n/2 on; bin n/2 is the negative
    Nyquist frequency for even n) times the bin spacing 1 / (n d).  Formed
    as index * spacing, so q is rounded the same way wherever it is formed:
    a metre-long free-space step turns q into phases of ~1e7 rad, where one
    ulp of q is already a phase error of ~1e-9."""
    m = np.arange(n)
    signed = np.where(m < (n + 1) // 2, m, m - n)
    return signed * (1.0 / (n * d))
