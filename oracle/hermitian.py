"""Stage B for Hermitian and positive semidefinite matrices (Section 5.3, 5.4) -- oracle side.

Test infrastructure only.

Given a symmetric A and a basis Q with ||A - Q Q^T A|| small (Stage A):
  * Algorithm 5.3, direct eigenvalue decomposition: B = Q^T A Q, B = V Lambda V^T,
    U = Q V.  A ~ U Lambda U^T with ||A - Q Q^T A Q Q^T|| <= 2 ||A - Q Q^T A|| (5.x).
  * Algorithm 5.5, the Nystrom method for psd A: B1 = A Q, B2 = Q^T B1 = C^T C
    (Cholesky, C upper), F = B1 C^-1 (triangular solve), F = U Sigma V^T,
    Lambda = Sigma^2; A ~ F F^T, whose spectral error never exceeds ||A - Q Q^T A||.
Eigenpairs are returned ordered by decreasing |lambda| and truncated to k (the Remark 5.1
truncation carried over); the sign of each eigenvector is not specified.

``operand`` (default: none) rounds the basis where it enters the product with A, B1 = A
operand(Q), for the tensor-core precision pattern (oracle.mixed.split: the basis as a
hi + lo pair of bfloat16 numbers); Q^T B1 and the lift U = Q V use Q itself.
"""
from __future__ import annotations

import numpy as np


def _b1(a, qmat, operand):
    return a @ (qmat if operand is None else operand(qmat))


def eig_direct(a: np.ndarray, qmat: np.ndarray, k: int, operand=None):
    """Algorithm 5.3.  Returns (U m x k, lambda k) by decreasing |lambda|."""
    b = qmat.T @ _b1(a, qmat, operand)
    b = 0.5 * (b + b.T)                  # B is symmetric; drop the rounding asymmetry
    lam, v = np.linalg.eigh(b)
    order = np.argsort(-np.abs(lam), kind="stable")[:k]
    return qmat @ v[:, order], lam[order]


def nystrom(a: np.ndarray, qmat: np.ndarray, k: int, operand=None):
    """Algorithm 5.5.  Returns (U m x k, lambda k >= 0, F m x l)."""
    b1 = _b1(a, qmat, operand)
    b2 = qmat.T @ b1
    b2 = 0.5 * (b2 + b2.T)
    c = np.linalg.cholesky(b2).T          # B2 = C^T C, C upper triangular
    f = np.linalg.solve(c.T, b1.T).T      # F = B1 C^-1
    u, s, _ = np.linalg.svd(f, full_matrices=False)
    return u[:, :k], (s * s)[:k], f
