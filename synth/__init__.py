"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module only builds input matrices; it contains none of the arithmetic of
the randomized range finder or SVD.  Every matrix is A = U diag(sigma) V^T with
U, V Haar-distributed orthonormal factors (QR of a seeded standard Gaussian
matrix with the column signs fixed so that diag(R) > 0, Mezzadri 2007) and a
prescribed spectrum sigma.  The paper's own test data (the FERET faces, the
image graph Laplacian, the integral operators of Section 7) are not available;
these spectra stand in for them, with the shapes of the workloads described in
the design notes.

Two back ends:
  * ``lowrank`` -- numpy float64 on the host, exact to rounding; used for every
    case the oracle solves in full.
  * ``device_lowrank`` -- torch on a CUDA device in float32, for the full-size
    workloads (16384^2 and up) where a host QR would take minutes.  The
    factors are orthonormal to float32 rounding, so the nominal sigma holds to
    about 1e-6 * sigma_1; parity checks always use the matrix as stored.
"""
from __future__ import annotations

import dataclasses

import numpy as np

# --------------------------------------------------------------------------
# spectra of the workloads
# --------------------------------------------------------------------------


def spectrum_exp(n: int, rate: float) -> np.ndarray:
    """sigma_j = exp(-(j-1)/rate), j = 1..n."""
    j = np.arange(n, dtype=np.float64)
    return np.exp(-j / rate)


def spectrum_power(n: int, power: float) -> np.ndarray:
    """sigma_j = j^(-power), j = 1..n."""
    j = np.arange(1, n + 1, dtype=np.float64)
    return j ** (-power)


def spectrum_exp_floor(n: int, rate: float, floor: float) -> np.ndarray:
    """sigma_j = max(exp(-(j-1)/rate), floor)."""
    return np.maximum(spectrum_exp(n, rate), floor)


# --------------------------------------------------------------------------
# host (float64) construction
# --------------------------------------------------------------------------


def haar(rng: np.random.Generator, n: int, k: int) -> np.ndarray:
    """n x k matrix with orthonormal columns, Haar distributed (k <= n)."""
    g = rng.standard_normal((n, k))
    q, r = np.linalg.qr(g)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d


def lowrank(m: int, n: int, sigma: np.ndarray, seed: int):
    """A = U diag(sigma) V^T in float64 with Haar U (m x r), V (n x r).

    ``sigma`` has r <= min(m, n) entries (r < min(m, n) gives an exactly
    rank-r matrix).  Returns (A, U, sigma, V).
    """
    sigma = np.asarray(sigma, dtype=np.float64)
    r = sigma.shape[0]
    rng = np.random.default_rng(seed)
    u = haar(rng, m, r)
    v = haar(rng, n, r)
    a = (u * sigma) @ v.T
    return a, u, sigma, v


def gaussian_matrix(rows: int, cols: int, seed: int) -> np.ndarray:
    """Plain seeded N(0,1) matrix (float64) for caller-supplied test matrices."""
    return np.random.default_rng(seed).standard_normal((rows, cols))


def noise(m: int, n: int, std: float, seed: int) -> np.ndarray:
    return std * np.random.default_rng(seed).standard_normal((m, n))


# --------------------------------------------------------------------------
# device (float32) construction for the full-size workloads
# --------------------------------------------------------------------------


def device_haar(n: int, k: int, generator, device):
    import torch

    g = torch.randn(n, k, generator=generator, device=device, dtype=torch.float32)
    q, r = torch.linalg.qr(g)
    d = torch.sign(torch.diagonal(r))
    d[d == 0] = 1.0
    return q * d


def device_lowrank(m: int, n: int, sigma: np.ndarray, seed: int, device="cuda",
                   noise_std: float = 0.0):
    """float32 A = U diag(sigma) V^T (+ iid N(0, noise_std^2)) built on a device."""
    import torch

    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        gen = torch.Generator(device=device)
        gen.manual_seed(int(seed))
        r = len(sigma)
        u = device_haar(m, r, gen, device)
        v = device_haar(n, r, gen, device)
        s = torch.as_tensor(np.asarray(sigma, dtype=np.float32), device=device)
        a = (u * s) @ v.T
        del u, v
        if noise_std > 0.0:
            a += noise_std * torch.randn(m, n, generator=gen, device=device,
                                         dtype=torch.float32)
        return a.contiguous()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    m: int
    n: int
    k: int
    p: int
    q: int
    spectrum: str          # human-readable recipe
    matrix_seed: int
    omega_seed: int

    @property
    def l(self) -> int:  # noqa: E743 - the paper's symbol
        return self.k + self.p

    def sigma(self) -> np.ndarray:
        r = min(self.m, self.n)
        if self.name == "c1":
            return spectrum_exp(r, 8.0)
        if self.name == "c2":
            return spectrum_power(r, 1.5)
        if self.name == "c3":
            return spectrum_exp_floor(r, 20.0, 1e-6)
        if self.name == "c4":
            return spectrum_power(r, 0.5)
        raise ValueError(self.name)

    def noise_std(self) -> float:
        return 1e-4 if self.name == "c3" else 0.0


C1 = Workload("c1", 2000, 1000, 20, 10, 2, "exp(-(j-1)/8)", 1001, 2001)
C2 = Workload("c2", 16384, 16384, 100, 10, 1, "j^-1.5", 1002, 2002)
C3 = Workload("c3", 262144, 4096, 64, 16, 2, "max(exp(-(j-1)/20),1e-6)+N(0,1e-8)", 1003, 2003)
C4 = Workload("c4", 32768, 32768, 236, 20, 1, "j^-0.5", 1004, 2004)

WORKLOADS = {w.name: w for w in (C1, C2, C3, C4)}

# Batched workload: 512 matrices, m ~ U[128, 2048], n ~ U[64, 1024] inclusive,
# sigma_j = exp(-(j-1)/4), k = 16, p = 8, q = 1.
C5_COUNT, C5_K, C5_P, C5_Q = 512, 16, 8, 1
C5_MATRIX_SEED, C5_OMEGA_SEED = 1005, 2005


def c5_shapes(seed: int = C5_MATRIX_SEED, count: int = C5_COUNT):
    rng = np.random.default_rng(seed)
    ms = rng.integers(128, 2048, size=count, endpoint=True)
    ns = rng.integers(64, 1024, size=count, endpoint=True)
    return [(int(a), int(b)) for a, b in zip(ms, ns)]


def c5_matrix(index: int, seed: int = C5_MATRIX_SEED):
    m, n = c5_shapes(seed)[index]
    return lowrank(m, n, spectrum_exp(min(m, n), 4.0), seed * 100003 + index)


def small_case(m: int, n: int, sigma: np.ndarray, seed: int):
    """Convenience alias used by tests for reduced-size versions of a workload."""
    return lowrank(m, n, sigma, seed)


def scaled_down(w: Workload, factor: int) -> Workload:
    """The same recipe at 1/factor of each dimension (tests that must stay fast)."""
    m = max(w.m // factor, 1)
    n = max(w.n // factor, 1)
    return dataclasses.replace(w, m=m, n=n, name=w.name)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even float64/float32 -> bfloat16 -> float64 (host model of a bf16 copy)."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = (b + 0x7FFF + lsb) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


__all__ = [
    "spectrum_exp", "spectrum_power", "spectrum_exp_floor", "haar", "lowrank",
    "gaussian_matrix", "noise", "device_lowrank", "Workload", "C1", "C2", "C3",
    "C4", "WORKLOADS", "c5_shapes", "c5_matrix", "small_case", "scaled_down",
    "bf16_round", "C5_COUNT", "C5_K", "C5_P", "C5_Q",
]
