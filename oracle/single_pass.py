"""Single-pass randomized SVD for a general matrix (Section 5.5) -- oracle side.

Test infrastructure only.

Steps as the paper lists them: draw Omega (n x l) and Psi (m x l'); form
Y = A Omega and Yt = A^T Psi in one pass over A; QR of both, Y = Q R and
Yt = Qt Rt; the reduced matrix B = Q^T A Qt satisfies
    Q^T Y  ~= B (Qt^T Omega)
    Qt^T Yt ~= B^T (Q^T Psi)
and is taken as the minimum-residual solution of both.

Reading (the paper leaves the solver open): minimise
    ||B X1 - C1||_F^2 + ||B^T X2 - C2||_F^2,
    X1 = Qt^T Omega, C1 = Q^T Y, X2 = Q^T Psi, C2 = Qt^T Yt,
whose normal equations are the Sylvester equation
    (X2 X2^T) B + B (X1 X1^T) = C1 X1^T + X2 C2^T,
solved exactly through the eigenbases of the two symmetric positive definite
matrices.  ``min_residual_bruteforce`` solves the same least-squares problem
through its Kronecker form, for tiny l only.

Bases (the remark on single-pass error in Section 5.5): with Q, Qt the full l-column
bases the coefficient matrices are square and usually ill-conditioned, and on noisy,
slowly decaying spectra the result degrades badly; the remark's remedy -- keep only
the k leading left singular vectors of each sample matrix, so that the systems above
are k x l, overdetermined -- is taken here (``truncate_bases=True``, the default);
with p = 0 both forms coincide.
"""
from __future__ import annotations

import numpy as np

from .rsvd64 import qr_pos, truncate


def two_sided_sketch(a: np.ndarray, omega: np.ndarray, psi: np.ndarray):
    return a @ omega, a.T @ psi


def reduced_system(qmat, qt, omega, psi, y, yt):
    x1 = qt.T @ omega
    c1 = qmat.T @ y
    x2 = qmat.T @ psi
    c2 = qt.T @ yt
    return x1, c1, x2, c2


def min_residual(x1, c1, x2, c2):
    p = x2 @ x2.T
    s = x1 @ x1.T
    rhs = c1 @ x1.T + x2 @ c2.T
    lp, up = np.linalg.eigh(p)
    ls, us = np.linalg.eigh(s)
    bh = (up.T @ rhs @ us) / (lp[:, None] + ls[None, :])
    return up @ bh @ us.T


def min_residual_bruteforce(x1, c1, x2, c2):
    """Least squares over vec(B) (column-major), for tiny problems."""
    l, lt = x2.shape[0], x1.shape[0]
    nb = l * lt
    rows = []
    rhs = []
    # B X1 = C1 : entry (i, j) = sum_t B[i, t] X1[t, j]
    for i in range(l):
        for j in range(x1.shape[1]):
            r = np.zeros(nb)
            for t in range(lt):
                r[i + t * l] = x1[t, j]
            rows.append(r)
            rhs.append(c1[i, j])
    # B^T X2 = C2 : entry (i, j) = sum_t B[t, i] X2[t, j]
    for i in range(lt):
        for j in range(x2.shape[1]):
            r = np.zeros(nb)
            for t in range(l):
                r[t + i * l] = x2[t, j]
            rows.append(r)
            rhs.append(c2[i, j])
    sol, *_ = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)
    return sol.reshape(lt, l).T


def leading_left(y: np.ndarray, k: int) -> np.ndarray:
    """The k leading left singular vectors of y."""
    return np.linalg.svd(y, full_matrices=False)[0][:, :k]


def rsvd_single_pass(a: np.ndarray, k: int, omega: np.ndarray, psi: np.ndarray,
                     truncate_bases: bool = True):
    """Rank-k factors (U, sigma, V) from one pass over A, plus (Q, Qt, B)."""
    y, yt = two_sided_sketch(a, omega, psi)
    if truncate_bases:
        qmat, qt = leading_left(y, k), leading_left(yt, k)
    else:
        qmat, _ = qr_pos(y)
        qt, _ = qr_pos(yt)
    x1, c1, x2, c2 = reduced_system(qmat, qt, omega, psi, y, yt)
    b = min_residual(x1, c1, x2, c2)
    ub, s, vbt = np.linalg.svd(b, full_matrices=False)
    u, s, v = truncate(qmat @ ub, s, qt @ vbt.T, k)
    return u, s, v, (qmat, qt, b)
