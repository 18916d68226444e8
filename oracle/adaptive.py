"""Adaptive randomized range finder for the fixed-precision problem (Section 4.4) -- oracle side.

Test infrastructure only.

Algorithm 4.2 grows an orthonormal basis Q one Gaussian sample at a time and stops once r
consecutive projected samples (I - Q Q^T) A w are shorter than eps / (10 sqrt(2/pi)): by
the posterior estimate (4.3) of Lemma 4.1, ||(I - Q Q^T) A|| <= eps then holds except with
probability min(m, n) 10^-r.  The remark after the algorithm organises the work in blocks
of samples; that is the form taken here (and on the GPU), with the block size b equal to
the number r of look-ahead samples the test uses:

  Y = A Omega_1                       (n x b block 1 of the sample stream)
  while max_i ||Y[:, i]|| > eps / (10 sqrt(2/pi))  and the basis has room for b more:
      Y <- (I - Q Q^T) Y              (step 7: reproject, the samples are unreliable once small)
      Q_blk = orth(Y)                 (QR, diag(R) > 0)
      Q_blk = orth((I - Q Q^T) Q_blk) (the normalised block reprojected, as the text after
                                       the algorithm describes for step 8: a sample at the
                                       rounding level keeps O(u ||y||) components along Q,
                                       which normalisation would blow up to O(1))
      Q <- [Q, Q_blk]
      Y <- (I - Q Q^T) A Omega_next   (steps 10-11 for the next block)
  return Q

Omega is the caller's n x (cap + b) matrix: block t is its columns (t-1) b .. t b - 1, so
both sides draw the same sample stream.  The stopping decision compares norms with the
threshold; the GPU takes it in float32, the oracle here in float64 (tests keep eps away
from the boundary).
"""
from __future__ import annotations

import numpy as np

from .rsvd64 import qr_pos

THRESHOLD_FACTOR = 10.0 * np.sqrt(2.0 / np.pi)   # the 10 sqrt(2/pi) of (4.3)


def project_out(qmat: np.ndarray, y: np.ndarray) -> np.ndarray:
    """(I - Q Q^T) y; Q may have no columns."""
    if qmat.shape[1] == 0:
        return y.copy()
    return y - qmat @ (qmat.T @ y)


def orth_block(qmat: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Steps 7-8 for a block: reproject y, orthonormalise, reproject the normalised block
    and orthonormalise it again (QR with diag(R) > 0 both times)."""
    qb, _ = qr_pos(project_out(qmat, y))
    qb, _ = qr_pos(project_out(qmat, qb))
    return qb


def adaptive_range_finder(a: np.ndarray, eps: float, omega: np.ndarray, block: int, cap: int):
    """Blocked Algorithm 4.2.  Returns (Q, est): Q m x j orthonormal (j a multiple of block,
    j <= cap) and est = max_i ||Y[:, i]|| of the last (unconsumed) test block."""
    m = a.shape[0]
    if omega.shape[1] < cap + block:
        raise ValueError("omega needs cap + block columns")
    qmat = np.zeros((m, 0))
    y = a @ omega[:, :block]
    t = 1
    while True:
        est = float(np.max(np.linalg.norm(y, axis=0)))
        if est <= eps / THRESHOLD_FACTOR or qmat.shape[1] + block > cap:
            return qmat, est
        qmat = np.hstack([qmat, orth_block(qmat, y)])
        y = project_out(qmat, a @ omega[:, t * block:(t + 1) * block])
        t += 1
