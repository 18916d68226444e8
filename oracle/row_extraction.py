"""Stage B by row extraction (Section 5.2, Algorithm 5.2) -- oracle side.

Test infrastructure only.

The interpolative decomposition (Section 3.2.3) of the rows of an m x l matrix Y of
rank l: an index set J of l rows and an m x l matrix X with X[J, :] = I and Y = X Y[J, :].
J comes from the classical device of Section 3.3.2, successive orthogonalization with
pivoting (Businger--Golub) applied to the rows: at each step the row whose residual is
longest is chosen, and its normalised residual is removed from every row.  X is then the
plain definition, X = Y Y[J, :]^-1 (a linear solve).

Algorithm 5.2 with the ID of the basis Q:
  1. Q = X Q[J, :]                     (the ID of the rows of Q)
  2. A[J, :] = R^T W^T                 (QR of A[J, :]^T = W R)
  3. Z = X R^T
  4. Z = U Sigma Vt^T                  (SVD)
  5. V = W Vt
so that U Sigma V^T = X A[J, :] (the identity in the proof of Lemma 5.1).  Everything is
returned untruncated (l columns); Remark 5.1's truncation to k is ``rsvd64.truncate``.

Readings: the algorithm takes Q (the unified presentation of Section 5) rather than the
sample matrix of the remark after Lemma 5.1; the pivoting is Businger--Golub, so the
entries of X are not guaranteed to stay below 2 (the bound the section quotes belongs to
the strong rank-revealing ID); Lemma 5.1's chain of inequalities holds for any X with
X[J, :] = I: ||A - U Sigma V^T|| <= (1 + ||X||) ||A - Q Q^T A||.  Ties in the pivot
choice go to the lowest row index.
"""
from __future__ import annotations

import numpy as np

from .rsvd64 import qr_pos


def pivot_rows(y: np.ndarray, count: int, with_margins: bool = False):
    """Businger--Golub pivoting on the rows of y: ``count`` row indices, in the order chosen.

    with_margins: also return, per step, how far the chosen row's squared residual norm
    stands above the next longest, relative to it (a decision that another rounding could
    take differently has a small margin)."""
    r = np.array(y, dtype=np.float64, copy=True)
    chosen: list[int] = []
    margins = []
    for _ in range(count):
        norms = np.einsum("ij,ij->i", r, r)
        norms[chosen] = -1.0
        j = int(np.argmax(norms))                # the first of equal maxima
        if with_margins:
            second = np.max(np.delete(norms, j)) if len(norms) > 1 else -1.0
            margins.append((norms[j] - max(second, 0.0)) / norms[j])
        chosen.append(j)
        v = r[j] / np.sqrt(norms[j])
        r -= np.outer(r @ v, v)
        r[j] = 0.0
    jset = np.array(chosen, dtype=np.int64)
    return (jset, np.array(margins)) if with_margins else jset


def interpolative_rows(y: np.ndarray):
    """ID of the rows of y (m x l, rank l): (J, X) with X[J] = I and y = X y[J]."""
    l = y.shape[1]
    jset = pivot_rows(y, l)
    x = np.linalg.solve(y[jset].T, y.T).T        # X y[J] = y
    x[jset] = np.eye(l)
    return jset, x


def svd_row_extraction(a: np.ndarray, qmat: np.ndarray):
    """Algorithm 5.2.  Returns (U m x l, sigma l, V n x l, J, X)."""
    jset, x = interpolative_rows(qmat)             # step 1
    w, r = qr_pos(a[jset].T)                       # step 2: A[J]^T = W R
    z = x @ r.T                                    # step 3
    u, s, vt_t = np.linalg.svd(z, full_matrices=False)   # step 4
    v = w @ vt_t.T                                 # step 5
    return u, s, v, jset, x
