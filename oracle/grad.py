"""Gradient of the rank-k reconstruction loss through the randomized SVD, Omega fixed -- oracle side.

Test infrastructure only.

Loss (the batched workload's training objective):
    L(A) = ||A - U_k S_k V_k^T||_F^2 + sum_{i<=k} sigma_i,
with (U_k, S_k, V_k) the output of the randomized SVD of A (Algorithm 4.4 as
Stage A, Algorithm 5.1 as Stage B, Remark 5.1 truncation) for a fixed test
matrix Omega.  The paper does not differentiate its algorithms; three
independent routes give the gradient here:
  * ``grad_fd``: central finite differences of ``loss`` in float64 (full for
    tiny matrices, or along given directions);
  * ``grad_autograd``: the same float64 steps written with torch CPU ops
    (LAPACK QR and SVD) and differentiated by torch's autograd;
  * ``grad_exact_svd``: the closed form 2 (A - A_k) + U_k V_k^T for the exact
    truncated SVD (d sigma_i = u_i^T dA v_i and ||A - A_k||_F^2 =
    ||A||_F^2 - sum_{i<=k} sigma_i^2), which the randomized gradient
    approaches when the basis captures the dominant subspace.

General cotangents (the library's rsvd_svd_backward takes any gU, gS, gV): the
gradient of <gU, U(A)> + <gS, S(A)> + <gV, V(A)> through the same map,
``cotangent_autograd`` (torch autograd of the float64 steps) and
``cotangent_fd`` (central differences, each singular pair's sign held to that
of the unperturbed A, so that U(A) and V(A) are the smooth branch being
differentiated).
"""
from __future__ import annotations

import numpy as np

from .rsvd64 import rsvd


def loss(a: np.ndarray, k: int, p: int, q: int, omega: np.ndarray) -> float:
    u, s, v, _ = rsvd(a, k, p, q, omega)
    r = a - (u * s) @ v.T
    return float(np.sum(r * r) + np.sum(s))


def grad_fd(a: np.ndarray, k: int, p: int, q: int, omega: np.ndarray, h: float = 1e-3,
            directions=None):
    """Central differences.  With ``directions`` (list of m x n arrays) returns the
    directional derivatives; otherwise the full m x n gradient."""
    if directions is not None:
        out = []
        for e in directions:
            fp = loss(a + h * e, k, p, q, omega)
            fm = loss(a - h * e, k, p, q, omega)
            out.append((fp - fm) / (2.0 * h))
        return np.array(out)
    g = np.zeros_like(a)
    for i in range(a.shape[0]):
        for j in range(a.shape[1]):
            e = np.zeros_like(a)
            e[i, j] = 1.0
            g[i, j] = (loss(a + h * e, k, p, q, omega) - loss(a - h * e, k, p, q, omega)) / (2.0 * h)
    return g


def grad_autograd(a: np.ndarray, k: int, p: int, q: int, omega: np.ndarray) -> np.ndarray:
    import torch

    at = torch.tensor(a, dtype=torch.float64, requires_grad=True)
    om = torch.tensor(omega, dtype=torch.float64)

    def qr_pos(y):
        qm, r = torch.linalg.qr(y, mode="reduced")
        d = torch.sign(torch.diagonal(r)).detach()
        d[d == 0] = 1.0
        return qm * d

    qm = qr_pos(at @ om)
    for _ in range(q):
        qt = qr_pos(at.T @ qm)
        qm = qr_pos(at @ qt)
    b = qm.T @ at
    ub, s, vbt = torch.linalg.svd(b, full_matrices=False)
    u = qm @ ub[:, :k]
    v = vbt[:k].T
    s = s[:k]
    r = at - (u * s) @ v.T
    val = (r * r).sum() + s.sum()
    val.backward()
    return at.grad.numpy().copy()


def grad_exact_svd(a: np.ndarray, k: int) -> np.ndarray:
    u, s, vt = np.linalg.svd(a, full_matrices=False)
    ak = (u[:, :k] * s[:k]) @ vt[:k]
    return 2.0 * (a - ak) + u[:, :k] @ vt[:k]


def _rsvd_torch(at, omega, k, q):
    """The float64 steps of ``loss`` (Algorithm 4.4 + 5.1) on a torch tensor."""
    import torch

    om = torch.tensor(omega, dtype=torch.float64)

    def qr_pos(y):
        qm, r = torch.linalg.qr(y, mode="reduced")
        d = torch.sign(torch.diagonal(r)).detach()
        d[d == 0] = 1.0
        return qm * d

    qm = qr_pos(at @ om)
    for _ in range(q):
        qt = qr_pos(at.T @ qm)
        qm = qr_pos(at @ qt)
    ub, s, vbt = torch.linalg.svd(qm.T @ at, full_matrices=False)
    return qm @ ub[:, :k], s[:k], vbt[:k].T


def cotangent_value(a, k, p, q, omega, gu, gs, gv, ref=None):
    """<gU, U> + <gS, S> + <gV, V> for the rank-k factors of ``rsvd`` on a; with ref =
    (U0, V0) each pair's sign is aligned to ref's (the branch through A0)."""
    u, s, v, _ = rsvd(a, k, p, q, omega)
    if ref is not None:
        d = np.sign(np.sum(u * ref[0], axis=0))
        d[d == 0] = 1.0
        u, v = u * d, v * d
    return float(np.sum(gu * u) + np.sum(gs * s) + np.sum(gv * v))


def cotangent_autograd(a, k, p, q, omega, gu, gs, gv):
    """Gradient of <gU, U> + <gS, S> + <gV, V> by torch autograd; returns (grad, U, S, V)."""
    import torch

    at = torch.tensor(a, dtype=torch.float64, requires_grad=True)
    u, s, v = _rsvd_torch(at, omega, k, q)
    val = (torch.tensor(gu) * u).sum() + (torch.tensor(gs) * s).sum() + (torch.tensor(gv) * v).sum()
    val.backward()
    return at.grad.numpy().copy(), u.detach().numpy(), s.detach().numpy(), v.detach().numpy()


def cotangent_fd(a, k, p, q, omega, gu, gs, gv, directions, h=1e-4, ref=None):
    """Central differences of ``cotangent_value`` along the given directions, on the sign
    branch of ref = (U0, V0) (default: the factors of ``rsvd`` at a)."""
    if ref is None:
        u0, _, v0, _ = rsvd(a, k, p, q, omega)
        ref = (u0, v0)
    out = []
    for e in directions:
        fp = cotangent_value(a + h * e, k, p, q, omega, gu, gs, gv, ref=ref)
        fm = cotangent_value(a - h * e, k, p, q, omega, gu, gs, gv, ref=ref)
        out.append((fp - fm) / (2.0 * h))
    return np.array(out)
