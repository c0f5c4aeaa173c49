"""Pins for the dense solve oracle (CPU only).

Independent references: the two-point system solved by hand, the C direct sum
(a separate code path for the same matrix), and two properties of the kernel:
complex symmetry of A, and positive semidefiniteness of Im(A) + k I (the kernel
sin(kr)/r, with its limit k on the diagonal, is the Fourier transform of the
uniform measure on the sphere |xi| = k, so every matrix of it is PSD).
"""
import math

import numpy as np

import synth
from oracle import direct, solve

K = 2.0 * math.pi


def test_two_point_system_closed_form():
    pts = np.array([[0.0, 0.0, 0.0], [0.2, 0.7, -0.4]])
    b = np.array([1.0 - 0.5j, 0.25 + 2.0j])
    sigma = 3.0 + 40.0j
    r = np.linalg.norm(pts[1] - pts[0])
    a = np.exp(1j * K * r) / r
    det = sigma * sigma - a * a
    ref = np.array([sigma * b[0] - a * b[1], sigma * b[1] - a * b[0]]) / det
    x = solve.solve_dense(pts, b, K, sigma)
    assert np.max(np.abs(x - ref)) < 1e-14 * np.max(np.abs(ref))


def test_matrix_matches_direct_sum_and_is_symmetric():
    pts = synth.sphere(300, 1.5, seed=21)
    pts[7] = pts[3]                                   # a coincident pair contributes nothing
    q = synth.complex_normal(22, 300)[0]
    A = solve.dense_matrix(pts, K)
    ref = direct.direct(pts, q, K)
    assert np.max(np.abs(A @ q - ref)) < 1e-12 * np.max(np.abs(ref))
    assert A[3, 7] == 0 and A[7, 3] == 0 and np.all(np.diag(A) == 0)
    assert np.array_equal(A, A.T)


def test_imaginary_part_plus_k_is_psd():
    pts = synth.sphere(400, 1.0, seed=23)
    A = solve.dense_matrix(pts, K)
    ev = np.linalg.eigvalsh(A.imag + K * np.eye(len(pts)))
    assert ev.min() > -1e-9 * ev.max()


def test_solution_residual_through_direct_sum():
    pts = synth.sphere(500, 1.5, seed=24)
    b = synth.complex_normal(25, 500)[0]
    for sigma in (100j, 20.0 + 60.0j):
        x = solve.solve_dense(pts, b, K, sigma)
        r = b - sigma * x - direct.direct(pts, x, K)
        assert np.linalg.norm(r) < 1e-11 * np.linalg.norm(b)


def _kappa(pts, sigma):
    A = solve.dense_matrix(pts, K)
    A[np.diag_indices_from(A)] += sigma
    sv = np.linalg.svd(A, compute_uv=False)
    return sv[0] / sv[-1]


def test_condition_numbers_behind_the_gpu_solve_bounds(sphere4k):
    """The GPU GMRES tests bound ||x - x*|| / ||x*|| by kappa ||r|| / ||b|| with kappa <= 10 on
    the 4,096-point sphere at sigma = 100i and kappa <= 25 on the three ellipsoid blocks of
    the batched test; check both bounds against an SVD of the dense matrix."""
    pts = sphere4k[0]
    assert _kappa(pts, 100j) <= 10.0
    geoms, sizes, _ = synth.ellipsoid_batch(3, seed=4101, nmin=800, nmax=2500, amin=0.8, amax=2.0)
    for g in geoms:
        assert _kappa(g, 100j) <= 25.0
