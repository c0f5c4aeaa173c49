"""Special functions for the oracle MLFMA, written out from their textbook definitions.

TEST INFRASTRUCTURE: this package is the CPU oracle.  Only the tests, the smoke
check and the benchmark's CPU-baseline leg may import it; the product path never does.

The paper leaves the mathematics of the five far-field stages to its references
(Sec. 2, "specific mathematical details are omitted").  The quantities here are
the standard ones behind them:

* Gauss-Legendre nodes/weights on [-1, 1]  (the theta quadrature of the sampling grid),
* spherical Bessel j_n (Miller downward recurrence, normalised by
  sum_n (2n+1) j_n(x)^2 = 1) and y_n (upward recurrence), h_n = j_n + i y_n,
* Legendre polynomials P_n (three-term recurrence),
* orthonormal associated Legendre functions Pbar_n^m with
  int_{-1}^{1} Pbar_n^m(x)^2 dx = 1 (standard column recurrence in n).

Pins (tests/test_oracle_special.py): numpy's leggauss, scipy's spherical_jn /
spherical_yn / lpmv, h_0(x) = -i e^{ix}/x, orthonormality under quadrature.
"""
from __future__ import annotations

import math

import numpy as np


def gauss_legendre(npts: int):
    """Nodes (ascending) and weights of the npts-point Gauss-Legendre rule.

    Newton iteration on P_npts starting from cos(pi (i - 1/4) / (npts + 1/2)).
    """
    if npts < 1:
        raise ValueError("npts >= 1")
    i = np.arange(1, npts + 1, dtype=np.float64)
    x = np.cos(math.pi * (i - 0.25) / (npts + 0.5))
    for _ in range(100):
        p0 = np.ones_like(x)
        p1 = x.copy()
        for n in range(1, npts):
            p0, p1 = p1, ((2 * n + 1) * x * p1 - n * p0) / (n + 1)
        # p1 = P_npts(x), p0 = P_{npts-1}(x)
        dp = npts * (x * p1 - p0) / (x * x - 1.0)
        dx = p1 / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p0 = np.ones_like(x)
    p1 = x.copy()
    for n in range(1, npts):
        p0, p1 = p1, ((2 * n + 1) * x * p1 - n * p0) / (n + 1)
    dp = npts * (x * p1 - p0) / (x * x - 1.0)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return x[order], w[order]


def spherical_jn_all(nmax: int, x: float) -> np.ndarray:
    """j_0(x) .. j_nmax(x) for one real x > 0 by Miller's downward recurrence.

    Recurrence j_{n-1} = (2n+1)/x j_n - j_{n+1}, started well above max(nmax, x)
    and normalised with the identity sum_{n>=0} (2n+1) j_n(x)^2 = 1.
    """
    x = float(x)
    if x == 0.0:
        out = np.zeros(nmax + 1)
        out[0] = 1.0
        return out
    nstart = int(max(nmax, x)) + 40 + int(2.0 * math.sqrt(max(nmax, x)))
    vals = np.zeros(nstart + 2)
    vals[nstart + 1] = 0.0
    vals[nstart] = 1.0
    for n in range(nstart, 0, -1):
        vals[n - 1] = (2 * n + 1) / x * vals[n] - vals[n + 1]
        if abs(vals[n - 1]) > 1e100:      # rescale so that squares stay finite
            vals[n - 1:] *= 1e-100
    s = np.sum((2.0 * np.arange(nstart + 2) + 1.0) * vals * vals)
    return vals[: nmax + 1] / math.sqrt(s)


def spherical_yn_all(nmax: int, x: float) -> np.ndarray:
    """y_0(x) .. y_nmax(x) by the upward recurrence from y_0 = -cos x / x."""
    x = float(x)
    out = np.zeros(nmax + 1)
    out[0] = -math.cos(x) / x
    if nmax >= 1:
        out[1] = -math.cos(x) / (x * x) - math.sin(x) / x
    for n in range(1, nmax):
        out[n + 1] = (2 * n + 1) / x * out[n] - out[n - 1]
    return out


def spherical_hn_all(nmax: int, x: float) -> np.ndarray:
    """Spherical Hankel functions of the first kind h_n = j_n + i y_n, n = 0..nmax."""
    return spherical_jn_all(nmax, x) + 1j * spherical_yn_all(nmax, x)


def legendre_all(nmax: int, t: np.ndarray) -> np.ndarray:
    """P_0(t) .. P_nmax(t), shape [nmax+1, *t.shape]."""
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros((nmax + 1,) + t.shape)
    out[0] = 1.0
    if nmax >= 1:
        out[1] = t
    for n in range(1, nmax):
        out[n + 1] = ((2 * n + 1) * t * out[n] - n * out[n - 1]) / (n + 1)
    return out


def assoc_legendre_normalized(nmax: int, m: int, x: np.ndarray) -> np.ndarray:
    """Pbar_n^m(x) for n = m .. nmax (rows), orthonormal on [-1, 1].

    Pbar_m^m = sqrt((2m+1)/2 * prod_{k=1..m} (2k-1)/(2k)) (1 - x^2)^{m/2}
    Pbar_{m+1}^m = x sqrt(2m+3) Pbar_m^m
    Pbar_n^m = a_nm (x Pbar_{n-1}^m - b_nm Pbar_{n-2}^m),
      a_nm = sqrt((4n^2 - 1) / (n^2 - m^2)),  b_nm = sqrt(((n-1)^2 - m^2) / (4 (n-1)^2 - 1)).
    The Condon-Shortley phase is omitted (every use is a product of two such values).
    Returns an array of shape [nmax - m + 1, len(x)].
    """
    x = np.asarray(x, dtype=np.float64)
    if m > nmax:
        return np.zeros((0,) + x.shape)
    s2 = np.maximum(1.0 - x * x, 0.0)
    c = 0.5 * (2 * m + 1)
    for kk in range(1, m + 1):
        c *= (2 * kk - 1) / (2 * kk)
    pmm = math.sqrt(c) * s2 ** (0.5 * m)
    out = np.zeros((nmax - m + 1,) + x.shape)
    out[0] = pmm
    if nmax >= m + 1:
        out[1] = x * math.sqrt(2 * m + 3) * pmm
    for n in range(m + 2, nmax + 1):
        a = math.sqrt((4.0 * n * n - 1.0) / (n * n - m * m))
        b = math.sqrt(((n - 1.0) ** 2 - m * m) / (4.0 * (n - 1.0) ** 2 - 1.0))
        out[n - m] = a * (x * out[n - m - 1] - b * out[n - m - 2])
    return out
