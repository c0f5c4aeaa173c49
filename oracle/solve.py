"""Dense reference for the iterative solve around the matvec.

TEST INFRASTRUCTURE (CPU oracle): only the tests, the smoke check and the
benchmark's CPU-baseline leg may use it.

Sec. 1 places the potential evaluation inside an iterative integral-equation
solver.  The system solved is (sigma I + A) x = b, where A is the matrix of the
potential (A_ij = e^{ik r_ij} / r_ij for i != j and r_ij > 0, zero otherwise:
the definition the MLFMA approximates) and sigma a complex diagonal term.  Its
solution is unique whenever sigma I + A is nonsingular, so the oracle is the
definition written out: build the dense matrix, then call a library LU solve.
No Krylov iteration is reproduced here; the GPU's GMRES iterate is compared
with this solution.

Parity status: pinned by tests/test_oracle_solve.py (two-point closed form,
complex symmetry, the matrix against the C direct sum, the residual of the
solution through the C direct sum).
"""
from __future__ import annotations

import numpy as np


def dense_matrix(points: np.ndarray, k: float) -> np.ndarray:
    """A[i, j] = e^{ik|r_i - r_j|} / |r_i - r_j| for i != j with r > 0, else 0 (complex128)."""
    p = np.asarray(points, dtype=np.float64)
    d = np.sqrt(((p[:, None, :] - p[None, :, :]) ** 2).sum(axis=2))
    A = np.zeros(d.shape, dtype=np.complex128)
    m = d > 0
    A[m] = np.exp(1j * k * d[m]) / d[m]
    return A


def solve_dense(points: np.ndarray, b: np.ndarray, k: float, sigma: complex) -> np.ndarray:
    """x with (sigma I + A) x = b, by LU (numpy.linalg.solve)."""
    A = dense_matrix(points, k)
    A[np.diag_indices_from(A)] += sigma
    return np.linalg.solve(A, np.asarray(b, dtype=np.complex128))
