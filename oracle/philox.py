"""Counter-based random numbers for the test matrices (oracle side).

Test infrastructure: only tests/, the smoke check and the bench's CPU-baseline
leg use this package.

The paper asks for a standard Gaussian test matrix (Section 4.1, Algorithm 4.1
step 1) and notes that the quality of the generator hardly matters.  Both the
CUDA path and this oracle draw it from the same counter-based generator, each
implemented independently from its published definition:

  Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
  as 1, 2, 3", SC'11): a 4 x 32-bit counter and a 2 x 32-bit key; each of the
  ten rounds multiplies counter words 0 and 2 by 0xD2511F53 and 0xCD9E8D57
  (64-bit products split into hi/lo halves) and mixes
      (c0, c1, c2, c3) -> (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0));
  between rounds the key is bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85).

  Uniforms: u = (2 * (x >> 9) + 1) * 2^-24, which lies in (0, 1), is exact in
  float32 and float64, and never reaches 0 or 1.

  Gaussians (Box and Muller 1958): z0 = sqrt(-2 ln u0) cos(2 pi u1),
  z1 = sqrt(-2 ln u0) sin(2 pi u1).

Element (i, j) of a rows x cols test matrix drawn with (seed, stream): let
g = j // 4, t = j % 4; (x0..x3) = Philox4x32-10(counter=(g, i, stream, 0),
key=(seed mod 2^32, seed // 2^32)); the pairs (u0, u1) and (u2, u3) give
(z0, z1) and (z2, z3); the element is z_t.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)

STREAM_OMEGA = 0        # Gaussian Omega (n x l)
STREAM_PSI = 1          # second test matrix of the two-sided single-pass sketch (m x l)
STREAM_SRFT = 2         # SRFT signs and sampled frequencies


def philox4x32_10(counter: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Vectorised Philox4x32-10.

    counter: (N, 4) uint32; key: (2,) or (N, 2) uint32.  Returns (N, 4) uint32.
    """
    c = np.asarray(counter, dtype=np.uint32).astype(np.uint64)
    k = np.broadcast_to(np.asarray(key, dtype=np.uint32), (c.shape[0], 2)).astype(np.uint64)
    c0, c1, c2, c3 = c[:, 0], c[:, 1], c[:, 2], c[:, 3]
    k0, k1 = k[:, 0].copy(), k[:, 1].copy()
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(W0)) & MASK32
            k1 = (k1 + np.uint64(W1)) & MASK32
        p0 = M0 * c0            # < 2^64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)


def seed_key(seed: int) -> np.ndarray:
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)


def bits_to_uniform(x: np.ndarray) -> np.ndarray:
    """(2 * (x >> 9) + 1) * 2^-24 in float64 (exact)."""
    x = np.asarray(x, dtype=np.uint32)
    return ((x >> np.uint32(9)).astype(np.float64) * 2.0 + 1.0) * 2.0 ** -24


def raw_words(seed: int, stream: int, rows: int, groups: int) -> np.ndarray:
    """Philox outputs for counters (g, i, stream, 0), g < groups, i < rows -> (rows, groups, 4)."""
    g = np.arange(groups, dtype=np.uint32)
    i = np.arange(rows, dtype=np.uint32)
    gg, ii = np.meshgrid(g, i)          # (rows, groups)
    ctr = np.zeros((rows * groups, 4), dtype=np.uint32)
    ctr[:, 0] = gg.ravel()
    ctr[:, 1] = ii.ravel()
    ctr[:, 2] = np.uint32(stream)
    out = philox4x32_10(ctr, seed_key(seed))
    return out.reshape(rows, groups, 4)


def gaussian(seed: int, stream: int, rows: int, cols: int) -> np.ndarray:
    """rows x cols standard Gaussian test matrix (float64 Box-Muller of the shared uniforms)."""
    if rows == 0 or cols == 0:
        return np.zeros((rows, cols))
    groups = (cols + 3) // 4
    w = raw_words(seed, stream, rows, groups)
    u = bits_to_uniform(w)               # (rows, groups, 4)
    r01 = np.sqrt(-2.0 * np.log(u[..., 0]))
    r23 = np.sqrt(-2.0 * np.log(u[..., 2]))
    t01 = 2.0 * np.pi * u[..., 1]
    t23 = 2.0 * np.pi * u[..., 3]
    z = np.stack([r01 * np.cos(t01), r01 * np.sin(t01),
                  r23 * np.cos(t23), r23 * np.sin(t23)], axis=-1)
    return z.reshape(rows, groups * 4)[:, :cols].copy()
