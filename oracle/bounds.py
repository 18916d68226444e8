"""Error bounds of the paper as plain formulas -- test infrastructure only.

Every function returns the right-hand side of one stated bound; tests compare
errors measured by the oracle against them.
"""
from __future__ import annotations

import math

import numpy as np


def intro_expectation(k: int, p: int, m: int, n: int, sigma_k1: float) -> float:
    """Theorem 1.1 (Section 1.5): E||A - QQ*A|| <= [1 + 4 sqrt(k+p)/(p-1) sqrt(min(m,n))] sigma_{k+1}."""
    return (1.0 + 4.0 * math.sqrt(k + p) / (p - 1) * math.sqrt(min(m, n))) * sigma_k1


def intro_probability(k: int, p: int, m: int, n: int, sigma_k1: float) -> float:
    """Probability bound stated after Theorem 1.1 (Section 1.5): ||A - QQ*A|| <= [1 + 11 sqrt(k+p) sqrt(min(m,n))] sigma_{k+1} w.p. >= 1 - 6 p^-p."""
    return (1.0 + 11.0 * math.sqrt(k + p) * math.sqrt(min(m, n))) * sigma_k1


def intro_probability_failure(p: int) -> float:
    return 6.0 * float(p) ** (-p)


def intro_rsvd_expectation(k: int, q: int, m: int, n: int, sigma_k1: float) -> float:
    """Theorem 1.2 (Section 1.6), rank-2k output of the power scheme."""
    return (1.0 + 4.0 * math.sqrt(2.0 * min(m, n) / (k - 1))) ** (1.0 / (2 * q + 1)) * sigma_k1


def avg_frobenius(k: int, p: int, sigma: np.ndarray) -> float:
    """Theorem 10.5: E||(I-P_Y)A||_F <= (1 + k/(p-1))^(1/2) (sum_{j>k} sigma_j^2)^(1/2)."""
    tail = np.sqrt(np.sum(np.asarray(sigma)[k:] ** 2))
    return math.sqrt(1.0 + k / (p - 1)) * tail


def avg_spectral(k: int, p: int, sigma: np.ndarray) -> float:
    """Theorem 10.6: E||(I-P_Y)A|| <= (1 + sqrt(k/(p-1))) sigma_{k+1} + e sqrt(k+p)/p (sum_{j>k} sigma_j^2)^(1/2)."""
    s = np.asarray(sigma)
    return (1.0 + math.sqrt(k / (p - 1))) * s[k] + math.e * math.sqrt(k + p) / p * math.sqrt(np.sum(s[k:] ** 2))


def avg_spectral_power(k: int, p: int, q: int, sigma: np.ndarray) -> float:
    """Corollary 10.10: bound on E||(I-P_Z)A|| for Z = (AA*)^q A Omega."""
    s = np.asarray(sigma, dtype=np.float64)
    e = 2 * q + 1
    inner = (1.0 + math.sqrt(k / (p - 1))) * s[k] ** e + math.e * math.sqrt(k + p) / p * math.sqrt(np.sum(s[k:] ** (2 * e)))
    return inner ** (1.0 / e)


def deterministic(sigma: np.ndarray, v: np.ndarray, omega: np.ndarray, k: int, norm: str = "2") -> float:
    """Theorem 9.1 right side (square root): (||S2||^2 + ||S2 Om2 Om1^+||^2)^(1/2).

    ``v`` holds all right singular vectors (n x r) and ``sigma`` all r singular
    values; Omega_1 = V_1^T Omega, Omega_2 = V_2^T Omega.
    """
    s = np.asarray(sigma)
    om1 = v[:, :k].T @ omega
    om2 = v[:, k:].T @ omega
    s2 = s[k:]
    t = (s2[:, None] * om2) @ np.linalg.pinv(om1)
    if norm == "2":
        a = s2[0] if s2.size else 0.0
        b = np.linalg.norm(t, 2) if t.size else 0.0
    else:
        a = np.sqrt(np.sum(s2 ** 2))
        b = np.linalg.norm(t, "fro")
    return float(math.sqrt(a * a + b * b))


def pinv_gauss_frobenius_mean(k: int, p: int) -> float:
    """Proposition 10.2: E||G^+||_F^2 = k / (p - 1) for a k x (k+p) standard Gaussian G."""
    return k / (p - 1)


def pinv_gauss_spectral_mean(k: int, p: int) -> float:
    """Proposition 10.2: E||G^+|| <= e sqrt(k+p) / p."""
    return math.e * math.sqrt(k + p) / p
