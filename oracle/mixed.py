"""The tensor-core precision pattern of the randomized SVD, in float64.

Test infrastructure only: imported by tests/, the smoke check and the bench's CPU
legs, never by the library.

The tensor-core form of the path forms every product with A on bfloat16 tensor
cores (float32 accumulation) and re-orthonormalises in float32.  The roundings this
introduces sit at fixed points of Algorithm 4.4 (Stage A) and Algorithm 5.1
(Stage B); everything else is the float64 computation of ``rsvd64``:

  * A enters every product as stored (the caller passes the stored matrix:
    bf16(A), or hi + lo = bf16(A) + bf16(A - bf16(A))), or, where only some products
    read the residual lo, as the stored hi in the others (a_last, a_final);
  * the operand of each product of Stage A -- Omega (Algorithm 4.4 step 2),
    Q_{j-1} (step 4), Qt_j (step 5) -- is rounded to bfloat16;
  * the product B^T = A^T Q of Algorithm 5.1 step 1 takes Q as the sum of two
    bfloat16 numbers, hi = bf16(Q) and lo = bf16(Q - hi) (16 significant bits);
  * the lift U = Q Ut (Algorithm 5.1 step 3) uses Q itself.

``bf16`` is round-to-nearest, ties-to-even, to 8 significant bits with the
exponent range of float32 (its subnormals included); it is written from that
definition, not from any library conversion.
"""
from __future__ import annotations

import numpy as np

from . import rsvd64


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 value (ties to even), returned as float64.

    x = f 2^e with f in [0.5, 1) (numpy.frexp); a bfloat16 number carries 8
    significant bits, so the spacing of its values near x is 2^(e - 8), and not
    finer than that of the subnormals, 2^-133 (the smallest normal is 2^-126).
    numpy.rint rounds halfway cases to the even multiple.
    """
    x = np.asarray(x, dtype=np.float64)
    _, e = np.frexp(x)
    ulp = np.ldexp(1.0, np.maximum(e, -125) - 8)
    return np.rint(x / ulp) * ulp


def split(x) -> np.ndarray:
    """hi + lo with hi = bf16(x), lo = bf16(x - hi): x to 16 significant bits."""
    hi = bf16(x)
    return hi + bf16(np.asarray(x, dtype=np.float64) - hi)


def range_finder(a_stored: np.ndarray, omega: np.ndarray, q: int, operand=None,
                 a_last: np.ndarray | None = None):
    """Algorithm 4.4 with the operand of every product rounded by ``operand`` (bf16).

    a_last: A as the last product of Stage A sees it (step 5 for j = q, step 2 for q = 0),
    the one whose sample becomes the final basis Q (default a_stored: every product sees
    the same stored A)."""
    operand = bf16 if operand is None else operand
    a_last = a_stored if a_last is None else a_last
    qj, _ = rsvd64.qr_pos((a_last if q == 0 else a_stored) @ operand(omega))
    for j in range(1, q + 1):
        qt, _ = rsvd64.qr_pos(a_stored.T @ operand(qj))
        qj, _ = rsvd64.qr_pos((a_last if j == q else a_stored) @ operand(qt))
    return qj


def rsvd(a_stored: np.ndarray, k: int, p: int, q: int, omega: np.ndarray,
         a_final: np.ndarray | None = None, operand=None, final_basis=None,
         a_last: np.ndarray | None = None):
    """Algorithm 4.4 + Algorithm 5.1 + Remark 5.1 under the tensor-core precision pattern.

    a_stored: A as the products of Stage A see it; a_last: A as the last of them sees it
    (default a_stored); a_final: A as B^T = A^T Q sees it (default a_stored).  operand /
    final_basis: the roundings of the Stage A operands and of Q in B^T = A^T Q (default
    bf16 and split; identity functions give rsvd64.rsvd).  Returns (U, sigma, V, Q)
    truncated to rank k.
    """
    l = k + p
    if omega.shape != (a_stored.shape[1], l):
        raise ValueError("omega must be n x (k+p)")
    a_final = a_stored if a_final is None else a_final
    final_basis = split if final_basis is None else final_basis
    qmat = range_finder(a_stored, omega, q, operand, a_last)
    b = (a_final.T @ final_basis(qmat)).T            # B = Q^T A with the split basis
    ut, s, vt = np.linalg.svd(b, full_matrices=False)
    u = qmat @ ut                                    # the lift uses Q itself
    return u[:, :k], s[:k], vt.T[:, :k], qmat
