"""FP64 reference of the randomized range finder and the direct SVD (Halko, Martinsson, Tropp).

Test infrastructure only (tests/, the smoke check, the bench's CPU baseline).

Each function follows one algorithm of the paper, step for step, in float64,
with LAPACK (numpy) for the dense QR and SVD of the steps that ask for "a QR
factorization" or "an SVD".  No blocking, fusion or reordering beyond what the
algorithms state.

Conventions fixed here (the paper leaves them open):
  * QR factors are normalised so that diag(R) >= 0; the orthonormal factor of
    a full-column-rank matrix is then unique, and it is the factor that a
    Cholesky-based QR produces in exact arithmetic.
  * Singular values are returned in descending order.
"""
from __future__ import annotations

import numpy as np


def qr_pos(y: np.ndarray):
    """Thin Householder QR y = Q R with diag(R) >= 0 (Algorithm 4.1 step 3)."""
    q, r = np.linalg.qr(y, mode="reduced")
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d, r * d[:, None]


def range_finder(a: np.ndarray, omega: np.ndarray, q: int = 0, keep_steps: bool = False):
    """Randomized subspace iteration (Algorithm 4.4); q = 0 is Algorithm 4.1.

    Step 2:  Y0 = A Omega,  Y0 = Q0 R0.
    Step 4:  Yt_j = A^T Q_{j-1} = Qt_j Rt_j.
    Step 5:  Y_j = A Qt_j = Q_j R_j.
    Step 7:  Q = Q_q.
    Returns Q, or (Q, steps) with every intermediate orthonormal factor in
    the order they are formed: [Q0, Qt1, Q1, Qt2, Q2, ...].
    """
    y = a @ omega
    qj, _ = qr_pos(y)
    steps = [qj]
    for _ in range(q):
        qt, _ = qr_pos(a.T @ qj)
        qj, _ = qr_pos(a @ qt)
        steps += [qt, qj]
    return (qj, steps) if keep_steps else qj


def power_iteration(a: np.ndarray, omega: np.ndarray, q: int):
    """Randomized power iteration (Algorithm 4.3): Y = (A A^T)^q A Omega, then QR.

    No orthonormalisation between the applications of A and A^T, so it loses
    the modes below eps^(1/(2q+1)) ||A|| (the round-off remark of Section 4.5); kept only as a check
    of the exact-arithmetic equivalence with Algorithm 4.4.
    """
    y = a @ omega
    for _ in range(q):
        y = a @ (a.T @ y)
    return qr_pos(y)[0]


def direct_svd(a: np.ndarray, qmat: np.ndarray):
    """Direct SVD (Algorithm 5.1): B = Q^T A, B = Ut S V^T, U = Q Ut.  Full rank of Q."""
    b = qmat.T @ a
    ut, s, vt = np.linalg.svd(b, full_matrices=False)
    return qmat @ ut, s, vt.T


def truncate(u: np.ndarray, s: np.ndarray, v: np.ndarray, k: int):
    """Remark 5.1: keep the k dominant singular triplets."""
    return u[:, :k], s[:k], v[:, :k]


def rsvd(a: np.ndarray, k: int, p: int, q: int, omega: np.ndarray):
    """Prototype randomized SVD with Algorithm 4.4 as Stage A and Algorithm 5.1 as Stage B.

    omega is the n x (k+p) test matrix (Algorithm 4.4 step 1 is the caller's
    draw, so the same Omega can be handed to both sides).  Returns the
    rank-k factors (U, sigma, V) and the basis Q.
    """
    l = k + p
    if omega.shape != (a.shape[1], l):
        raise ValueError("omega must be n x (k+p)")
    qmat = range_finder(a, omega, q)
    u, s, v = direct_svd(a, qmat)
    u, s, v = truncate(u, s, v, k)
    return u, s, v, qmat


def rsvd_via_qr_of_bt(a: np.ndarray, k: int, p: int, q: int, omega: np.ndarray,
                      small_svd=None):
    """Same result as ``rsvd``, with Stage B's SVD taken as in Section 3.3.3.

    B^T = A^T Q is factored B^T = Q_B R_B, the ell x ell matrix R_B^T gets an
    SVD R_B^T = Ut S Wt^T, and U = Q Ut, V = Q_B Wt (B = R_B^T Q_B^T).
    ``small_svd`` defaults to LAPACK; tests pass the Jacobi SVD of
    oracle.jacobi to cross-check it.
    """
    qmat = range_finder(a, omega, q)
    bt = a.T @ qmat
    qb, rb = qr_pos(bt)
    if small_svd is None:
        ut, s, wtt = np.linalg.svd(rb.T)
        wt = wtt.T
    else:
        ut, s, wt = small_svd(rb.T)
    u = qmat @ ut
    v = qb @ wt
    return u[:, :k], s[:k], v[:, :k], qmat
