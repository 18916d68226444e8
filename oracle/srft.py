"""Subsampled random Fourier transform test matrix (Section 4.6) -- oracle side.

Test infrastructure only.

Omega = sqrt(n / l) * D F R with D diagonal random, F the unitary n-point DFT
(f_pq = n^(-1/2) exp(-2 pi i (p-1)(q-1) / n)) and R a sampling of l columns
without replacement (Algorithm 4.5 step 1).

Readings taken here (the paper is general; the workload fixes the rest):
  * D has random +-1 entries (the workload asks for random signs; the paper's
    unit-circle phases reduce to this for a real D).
  * A is real, so the columns of A D F at frequencies b and n-b are complex
    conjugates.  The l_c sampled frequencies are drawn without replacement from
    {1, ..., n/2 - 1} (one representative per conjugate pair, excluding the
    self-conjugate frequencies 0 and n/2), and the real sketch is
    [Re y_1, Im y_1, Re y_2, Im y_2, ...], m x 2 l_c, which spans the same real
    space as the complex samples at frequencies b_c and n - b_c.  "l" real
    columns therefore means l_c = l / 2 sampled frequencies.
  * Draws (Philox4x32-10, stream 2; see oracle.philox):
      sign d_i: word (i mod 4) of Philox(counter=(i div 4, 0, 2, 0)); d_i = -1
      when its top bit is set, else +1.
      frequencies: each candidate b in {1..n/2-1} gets the key word (b mod 4)
      of Philox(counter=(b div 4, 1, 2, 0)); the l_c candidates with the
      smallest (key, b) are taken, in that ascending order.
"""
from __future__ import annotations

import numpy as np

from .philox import STREAM_SRFT, philox4x32_10, seed_key


def _words(seed: int, row: int, count: int) -> np.ndarray:
    groups = (count + 3) // 4
    ctr = np.zeros((groups, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(groups, dtype=np.uint32)
    ctr[:, 1] = np.uint32(row)
    ctr[:, 2] = np.uint32(STREAM_SRFT)
    return philox4x32_10(ctr, seed_key(seed)).reshape(-1)[:count]


def draw(seed: int, n: int, lc: int):
    """Return (signs (n,) float64 +-1, freqs (lc,) int64) for an SRFT of length n."""
    if n % 2 or n < 4:
        raise ValueError("n must be even and >= 4")
    if lc > n // 2 - 1:
        raise ValueError("too many sampled frequencies")
    w = _words(seed, 0, n)
    signs = np.where(w >> np.uint32(31), -1.0, 1.0)
    cand = np.arange(1, n // 2, dtype=np.int64)
    keys = _words(seed, 1, n // 2)[cand]          # key of b is word b of row 1
    order = np.lexsort((cand, keys.astype(np.int64)))
    return signs, cand[order[:lc]]


def dft_matrix(n: int) -> np.ndarray:
    """Unitary DFT, f_pq = n^(-1/2) exp(-2 pi i p q / n), 0-based indices."""
    idx = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(idx, idx) / n) / np.sqrt(n)


def omega_complex(signs: np.ndarray, freqs: np.ndarray) -> np.ndarray:
    """Explicit n x l_c complex SRFT: sqrt(n / l_c) D F R (brute force, small n only)."""
    n = signs.shape[0]
    lc = freqs.shape[0]
    f = dft_matrix(n)[:, freqs]
    return np.sqrt(n / lc) * signs[:, None] * f


def omega_real(signs: np.ndarray, freqs: np.ndarray) -> np.ndarray:
    """n x 2 l_c real test matrix with interleaved columns [Re w_1, Im w_1, ...]."""
    n = signs.shape[0]
    lc = freqs.shape[0]
    idx = np.arange(n)[:, None]
    ang = -2.0 * np.pi * (idx * freqs[None, :] % n) / n
    scale = np.sqrt(n / lc) / np.sqrt(n)
    out = np.empty((n, 2 * lc))
    out[:, 0::2] = scale * signs[:, None] * np.cos(ang)
    out[:, 1::2] = scale * signs[:, None] * np.sin(ang)
    return out


def sketch_fft(a: np.ndarray, signs: np.ndarray, freqs: np.ndarray) -> np.ndarray:
    """Y = A Omega via a full FFT of each row of A D (Algorithm 4.5 step 2, full-FFT form)."""
    n = a.shape[1]
    lc = freqs.shape[0]
    yc = np.fft.fft(a * signs[None, :], axis=1, norm="ortho")[:, freqs] * np.sqrt(n / lc)
    out = np.empty((a.shape[0], 2 * lc))
    out[:, 0::2] = yc.real
    out[:, 1::2] = yc.imag
    return out


# ---- the modified SRFT with chains of random Givens rotations (Section 4.6, eq. random_Givens)
#
# Omega = D'' Theta' D' Theta (sqrt(n / l_c) D F R): the SRFT above with an orthogonal
# factor on the left, Theta = Pi G(1, 2; t_1) G(2, 3; t_2) ... G(n-1, n; t_{n-1}).
# Readings: the rotations are real (A is real; D, D', D'' are +-1 like D) with the
# convention of the cited Golub--Van Loan section, G(i, j; t) = I except
# [[c, s], [-s, c]] in rows and columns (i, j), c = cos t, s = sin t; Pi is the
# permutation (Pi x)_t = x_perm[t]; the scale sqrt(n / l_c) of the SRFT is kept (the
# remark leaves it out; a scale does not change the range).
# Draws (Philox4x32-10, stream 2, word i mod 4 of counter (i div 4, row, 2, 0)):
#   row 2: d'_i (top bit set: -1)     row 3: d''_i
#   row 4: keys of Pi: perm lists 0..n-1 by ascending (key, index)
#   row 5: t_i = 2 pi u_i, u_i = (word >> 8) 2^-24, for the rotation in plane (i, i+1)
#   rows 6, 7: the same for Pi', t'.

def gsrft_draw(seed: int, n: int):
    """Return (d1, d2 (n,) +-1, perm1, perm2 (n,) int64, theta1, theta2 (n - 1,) angles)."""
    def signs(row):
        return np.where(_words(seed, row, n) >> np.uint32(31), -1.0, 1.0)

    def perm(row):
        keys = _words(seed, row, n).astype(np.int64)
        return np.lexsort((np.arange(n), keys))

    def angles(row):
        u = (_words(seed, row, n - 1) >> np.uint32(8)).astype(np.float64) * 2.0 ** -24
        return 2.0 * np.pi * u

    return signs(2), signs(3), perm(4), perm(6), angles(5), angles(7)


def givens_chain(theta: np.ndarray, x: np.ndarray) -> np.ndarray:
    """G(1, 2; t_1) ... G(n-1, n; t_{n-1}) x for x (n,) or (n, cols): the rightmost
    rotation acts first."""
    y = np.array(x, dtype=np.float64, copy=True)
    for i in range(len(theta) - 1, -1, -1):
        c, s = np.cos(theta[i]), np.sin(theta[i])
        yi, yj = y[i].copy(), y[i + 1].copy()
        y[i] = c * yi + s * yj
        y[i + 1] = -s * yi + c * yj
    return y


def gsrft_omega_real(seed: int, n: int, lc: int) -> np.ndarray:
    """n x 2 l_c real modified SRFT: D'' Theta' D' Theta applied to the columns of the
    real SRFT of the same seed."""
    d, f = draw(seed, n, lc)
    d1, d2, p1, p2, t1, t2 = gsrft_draw(seed, n)
    w = omega_real(d, f)
    w = givens_chain(t1, w)[p1]          # Theta = Pi G(1, 2) ... G(n-1, n)
    w = d1[:, None] * w                  # D'
    w = givens_chain(t2, w)[p2]          # Theta'
    return d2[:, None] * w               # D''
