"""Pins for the oracle's special functions (CPU only).

Each function is compared with an independent library routine or a closed form,
never with a re-typed copy of its own formula.
"""
import math

import numpy as np
import pytest
import scipy.special as sp

from oracle import special


@pytest.mark.parametrize("n", [1, 2, 3, 9, 14, 21, 34, 58, 105, 197, 209])
def test_gauss_legendre_matches_numpy(n):
    x, w = special.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.max(np.abs(x - xr)) < 1e-13
    assert np.max(np.abs(w - wr)) < 1e-13 * max(1.0, np.max(wr))
    assert abs(w.sum() - 2.0) < 1e-13


def test_gauss_legendre_exact_on_even_monomials():
    x, w = special.gauss_legendre(12)
    for p in range(0, 24, 2):            # exact up to degree 2n-1 = 23
        assert abs(np.sum(w * x ** p) - 2.0 / (p + 1)) < 1e-14


@pytest.mark.parametrize("x", [1e-3, 0.3, 1.0, 3.14159, 7.5, 25.0, 101.3, 522.0])
def test_spherical_jn_yn_match_scipy(x):
    nmax = 250
    n = np.arange(nmax + 1)
    j = special.spherical_jn_all(nmax, x)
    jr = sp.spherical_jn(n, x)
    assert np.max(np.abs(j - jr)) <= 1e-12 * np.max(np.abs(jr))
    y = special.spherical_yn_all(nmax, x)
    yr = sp.spherical_yn(n, x)
    ok = np.isfinite(yr) & (np.abs(yr) < 1e300)
    rel = np.abs(y[ok] - yr[ok]) / np.maximum(np.abs(yr[ok]), 1e-300)
    # y_n is the dominant solution: relative accuracy wherever it is finite
    assert np.max(rel) < 1e-10


@pytest.mark.parametrize("x", [0.2, 1.0, 5.0, 40.0])
def test_h0_closed_form(x):
    h = special.spherical_hn_all(3, x)
    assert abs(h[0] - (-1j * np.exp(1j * x) / x)) < 1e-14 / x


def test_legendre_matches_scipy():
    t = np.linspace(-1, 1, 101)
    P = special.legendre_all(60, t)
    for n in (0, 1, 2, 7, 30, 60):
        assert np.max(np.abs(P[n] - sp.eval_legendre(n, t))) < 1e-12


@pytest.mark.parametrize("m", [0, 1, 2, 5, 11])
def test_assoc_legendre_matches_lpmv(m):
    nmax = 25
    x = np.linspace(-0.99, 0.99, 41)
    Pb = special.assoc_legendre_normalized(nmax, m, x)
    for n in range(m, nmax + 1):
        norm = math.sqrt((2 * n + 1) / 2.0 * math.factorial(n - m) / math.factorial(n + m))
        ref = sp.lpmv(m, n, x) * norm
        # the oracle drops the Condon-Shortley phase (-1)^m
        assert np.max(np.abs(Pb[n - m] - (-1) ** m * ref)) < 1e-11 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("L", [8, 40, 120])
def test_assoc_legendre_orthonormal_under_quadrature(L):
    x, w = special.gauss_legendre(L + 1)
    for m in (0, 1, L // 3, L - 1, L):
        Pb = special.assoc_legendre_normalized(L, m, x)
        G = (Pb * w[None, :]) @ Pb.T
        assert np.max(np.abs(G - np.eye(G.shape[0]))) < 1e-12
