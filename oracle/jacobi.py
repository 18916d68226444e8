"""One-sided (Hestenes) Jacobi SVD in float64 -- oracle cross-check of the small SVD.

Test infrastructure only.

Algorithm 5.1 step 2 asks for "an SVD of the small matrix" B.  LAPACK is the
primary oracle for it; this plain one-sided Jacobi (Hestenes 1958; the
rotation angle as in Rutishauser's formulation) is a second, independent
route, checked against LAPACK on small inputs.  It orthogonalises the columns
of X by plane rotations X <- X J(i, j, theta) until every pair is orthogonal
to working precision; then sigma_c = ||x_c||, u_c = x_c / sigma_c and V = the
accumulated rotations, so X = U diag(sigma) V^T.
"""
from __future__ import annotations

import numpy as np


def jacobi_svd(x: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """Return (U, sigma, V) of a square or tall matrix x (n_rows >= n_cols), sigma descending."""
    x = np.array(x, dtype=np.float64, copy=True)
    n = x.shape[1]
    v = np.eye(n)
    for _ in range(max_sweeps):
        rotated = False
        for i in range(n - 1):
            for j in range(i + 1, n):
                alpha = x[:, i] @ x[:, i]
                beta = x[:, j] @ x[:, j]
                gamma = x[:, i] @ x[:, j]
                if gamma == 0.0 or abs(gamma) <= tol * np.sqrt(alpha * beta):
                    continue
                rotated = True
                zeta = (beta - alpha) / (2.0 * gamma)
                t = np.sign(zeta) / (abs(zeta) + np.sqrt(1.0 + zeta * zeta)) if zeta != 0 else 1.0
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = c * t
                xi, xj = x[:, i].copy(), x[:, j].copy()
                x[:, i] = c * xi - s * xj
                x[:, j] = s * xi + c * xj
                vi, vj = v[:, i].copy(), v[:, j].copy()
                v[:, i] = c * vi - s * vj
                v[:, j] = s * vi + c * vj
        if not rotated:
            break
    sigma = np.sqrt(np.sum(x * x, axis=0))
    order = np.argsort(-sigma, kind="stable")
    sigma = sigma[order]
    x = x[:, order]
    v = v[:, order]
    u = np.zeros_like(x)
    nz = sigma > 0
    u[:, nz] = x[:, nz] / sigma[nz]
    return u, sigma, v
