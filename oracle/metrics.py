"""Error measures and comparison helpers (float64) -- test infrastructure only."""
from __future__ import annotations

import numpy as np


def fro_error(a: np.ndarray, u: np.ndarray, s: np.ndarray, v: np.ndarray) -> float:
    """||A - U diag(s) V^T||_F computed directly."""
    r = np.asarray(a, dtype=np.float64) - (u * s) @ v.T
    return float(np.sqrt(np.sum(r * r)))


def fro_error_onepass(a: np.ndarray, u: np.ndarray, s: np.ndarray, v: np.ndarray) -> float:
    """||A - U S V^T||_F^2 = ||A||_F^2 - 2 sum_i s_i u_i^T A v_i + ||U S V^T||_F^2 (one read of A)."""
    a = np.asarray(a, dtype=np.float64)
    cross = np.einsum("ij,ij->j", u, a @ v)
    low = (u * s).T @ (u * s)
    vv = v.T @ v
    e2 = np.sum(a * a) - 2.0 * np.sum(s * cross) + np.sum(low * vv)
    return float(np.sqrt(max(e2, 0.0)))


def spec_norm(mat: np.ndarray, iters: int = 0, seed: int = 0) -> float:
    """Spectral norm: dense SVD, or ``iters`` steps of power iteration on M^T M."""
    if iters <= 0:
        return float(np.linalg.norm(mat, 2))
    x = np.random.default_rng(seed).standard_normal(mat.shape[1])
    x /= np.linalg.norm(x)
    val = 0.0
    for _ in range(iters):
        y = mat.T @ (mat @ x)
        val = np.linalg.norm(y)
        if val == 0:
            return 0.0
        x = y / val
    return float(np.sqrt(val))


def projection_error(a: np.ndarray, qmat: np.ndarray, norm: str = "2") -> float:
    """||(I - Q Q^T) A|| in the spectral ('2') or Frobenius ('fro') norm."""
    r = a - qmat @ (qmat.T @ a)
    return float(np.linalg.norm(r, 2 if norm == "2" else "fro"))


def orthonormality(qmat: np.ndarray) -> float:
    """max |Q^T Q - I|."""
    g = qmat.T @ qmat
    return float(np.max(np.abs(g - np.eye(g.shape[0]))))


def align_columns(ref: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Flip the sign of each column of x to agree with ref (singular vectors are sign-free)."""
    d = np.sign(np.sum(ref * x, axis=0))
    d[d == 0] = 1.0
    return x * d


def canonical_signs(u: np.ndarray, v: np.ndarray):
    """Fix the sign of each singular pair so the largest-|.| entry of v_j is positive."""
    idx = np.argmax(np.abs(v), axis=0)
    d = np.sign(v[idx, np.arange(v.shape[1])])
    d[d == 0] = 1.0
    return u * d, v * d


def gap_bound(s: np.ndarray, eps: float, c: float = 1.0, s_next: float | None = None) -> np.ndarray:
    """Per-column Wedin-style bound c * eps * sigma_1 / gap_j on ||x_j - x_j'||.

    gap_j = min(sigma_{j-1} - sigma_j, sigma_j - sigma_{j+1}); the last column
    uses ``s_next`` (sigma_{k+1} of the reference) when given.
    """
    s = np.asarray(s, dtype=np.float64)
    k = s.shape[0]
    gaps = np.full(k, np.inf)
    for j in range(k):
        g = np.inf
        if j > 0:
            g = min(g, s[j - 1] - s[j])
        if j + 1 < k:
            g = min(g, s[j] - s[j + 1])
        elif s_next is not None:
            g = min(g, s[j] - s_next)
        gaps[j] = g
    return np.minimum(c * eps * s[0] / np.maximum(gaps, 1e-300), 2.0)
