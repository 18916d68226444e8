"""GPU parity of the backward passes (Omega held fixed) against the float64 oracle.

rsvd_svd_backward (one matrix, any cotangents gU, gS, gV, optionally the reconstruction
loss ||A - U S V^T||_F^2 + sum S) is compared with torch autograd through the oracle's
float64 steps of Algorithm 4.4 + 5.1 (oracle.grad, pinned against central differences),
on the sign branch of the GPU's factors (each cotangent column is flipped with its
singular pair).  Tolerance, as for the batched backward: the gradient passes through
R_0^-T and the SVD adjoint, so float32 rounding is amplified by kappa(Y_0) = kappa(R_0):
    ||gA - gA_ref||_F / ||gA_ref||_F <= 1e-4 + 20 u32 kappa(Y_0).
The batched backward is checked against central differences of the oracle's loss
(h = 1e-3, float64) along random directions on the first 8 matrices of the 512-matrix
workload.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import grad, philox

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _np(t):
    return t.detach().double().cpu().numpy()


def _signs(u, u_ref):
    d = np.sign(np.sum(u * u_ref, axis=0))
    d[d == 0] = 1.0
    return d


def _case(m, n, seed):
    sig = np.exp(-np.arange(min(m, n)) / 3.0) + 1e-3 * np.exp(-np.arange(min(m, n)) / 50.0)
    a, *_ = synth.lowrank(m, n, sig, seed)
    return a.astype(np.float32)


@pytest.mark.parametrize("m,n,k,p,q,recompute", [(300, 200, 10, 6, 1, 0), (300, 200, 10, 6, 1, 1),
                                                 (257, 390, 12, 4, 2, 0), (257, 390, 12, 4, 2, 1),
                                                 (400, 300, 16, 8, 0, 0), (1100, 700, 40, 24, 1, 0)])
def test_backward_cotangents_fp32(rsvd_lib, m, n, k, p, q, recompute):
    pkg = rsvd_lib
    a32 = _case(m, n, m + n)
    a64 = a32.astype(np.float64)
    rng = np.random.default_rng(m * n + q)
    gu, gs, gv = rng.standard_normal((m, k)), rng.standard_normal(k), rng.standard_normal((n, k))
    seed = 11
    om = philox.gaussian(seed, philox.STREAM_OMEGA, n, k + p)
    g_ref, u_ref, _, _ = grad.cotangent_autograd(a64, k, p, q, om, gu, gs, gv)
    with pkg.Plan(m, n, k, p, q, seed, recompute=recompute) as pl:
        A = torch.tensor(a32, device="cuda")
        U, S, V = pl.svd(A)
        d = _signs(_np(U), u_ref)
        dev = lambda x: torch.tensor(x, dtype=torch.float32, device="cuda")  # noqa: E731
        g = _np(pl.backward(A, dev(gu * d), dev(gs), dev(gv * d)))
        g2 = _np(pl.backward(A, dev(gu * d), dev(gs), dev(gv * d)))   # repeatable
    rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    kap = np.linalg.cond(a64 @ om)
    tol = 1e-4 + 20 * U32 * kap
    print(f"cotangent backward {m}x{n} k={k} q={q} recompute={recompute}: rel {rel:.3e} tol {tol:.3e}")
    assert rel <= tol
    assert np.array_equal(g, g2)


@pytest.mark.parametrize("recompute", [0, 1])
def test_backward_reconstruction_loss_fp32(rsvd_lib, recompute):
    """add_recon = 1 with no cotangents: the gradient of ||A - U S V^T||_F^2 + sum S."""
    pkg = rsvd_lib
    m, n, k, p, q, seed = 500, 380, 14, 6, 1, 3
    a32 = _case(m, n, 9)
    om = philox.gaussian(seed, philox.STREAM_OMEGA, n, k + p)
    g_ref = grad.grad_autograd(a32.astype(np.float64), k, p, q, om)
    with pkg.Plan(m, n, k, p, q, seed, recompute=recompute) as pl:
        A = torch.tensor(a32, device="cuda")
        pl.svd(A)
        g = _np(pl.backward(A, add_recon=1))
    rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    tol = 1e-4 + 20 * U32 * np.linalg.cond(a32.astype(np.float64) @ om)
    print(f"recon backward recompute={recompute}: rel {rel:.3e} tol {tol:.3e}")
    assert rel <= tol


def test_autograd_function_matches_builtin_loss(rsvd_lib):
    """The torch.autograd.Function: the loss written in torch on (U, S, V) gives the same
    A.grad as the library's built-in reconstruction loss."""
    pkg = rsvd_lib
    m, n, k, p, q = 420, 333, 12, 8, 1
    a32 = _case(m, n, 5)
    with pkg.Plan(m, n, k, p, q, 4) as pl:
        A = torch.tensor(a32, device="cuda", requires_grad=True)
        U, S, V = pkg.svd_autograd(A, pl)
        loss = ((A - (U * S) @ V.T) ** 2).sum() + S.sum()
        loss.backward()
        g_fn = _np(A.grad)
        pl.svd(A.detach())
        g_lib = _np(pl.backward(A.detach(), add_recon=1))
    rel = np.linalg.norm(g_fn - g_lib) / np.linalg.norm(g_lib)
    assert rel <= 1e-3, rel


@pytest.mark.parametrize("dtype", ["bf16", "hilo"])
def test_backward_tensor_cores(rsvd_lib, dtype):
    """Tensor-core plans: the backward passes carry their float32 operands as bfloat16 hi +
    lo pairs, but the forward's Stage A rounds its operands Q_j to bfloat16 (relative
    2^-9 per entry), so the bases the backward runs through differ from the oracle's
    (same stored A, same bfloat16-exact Omega) by that much, and the gradient inherits
    it: ||gA - gA_ref||_F / ||gA_ref||_F <= 2^-9."""
    pkg = rsvd_lib
    m, n, k, p, q, seed = 640, 512, 16, 8, 1, 21
    a32 = _case(m, n, 17)
    rng = np.random.default_rng(3)
    om = philox.gaussian(seed, philox.STREAM_OMEGA, n, k + p)
    om_b = torch.tensor(om, dtype=torch.float32).to(torch.bfloat16).float()
    gu, gs, gv = rng.standard_normal((m, k)), rng.standard_normal(k), rng.standard_normal((n, k))
    kw = dict(dtype=pkg.RSVD_BF16X2, residual_passes=1) if dtype == "hilo" else {}
    with pkg.Plan(m, n, k, p, q, seed, pkg.RSVD_BF16_TC, **kw) as pl:
        A = pl.stored(torch.tensor(a32, device="cuda"))
        pkg.rsvd_set_omega(pl.handle, om_b.cuda())
        U, S, V = pl.svd(A)
        a_st = _np(A)
        a_st = a_st[:m] + a_st[m:] if dtype == "hilo" else a_st
        g_ref, u_ref, _, _ = grad.cotangent_autograd(a_st, k, p, q, om_b.double().numpy(), gu, gs, gv)
        d = _signs(_np(U), u_ref)
        dev = lambda x: torch.tensor(x, dtype=torch.float32, device="cuda")  # noqa: E731
        g = _np(pl.backward(A, dev(gu * d), dev(gs), dev(gv * d)))
    rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    tol = 2.0 ** -9
    print(f"tensor-core backward {dtype}: rel {rel:.3e} tol {tol:.3e}")
    assert rel <= tol


def test_batched_backward_finite_differences_c5(rsvd_lib):
    """The first 8 matrices of the batched workload: <dL/dA_b, E> against central
    differences of the oracle's float64 loss (h = 1e-3) on the same bfloat16 A_b and
    bfloat16 Omega_b, four random unit directions per matrix."""
    pkg = rsvd_lib
    shapes = synth.c5_shapes()[:8]
    k, p, q, seed = synth.C5_K, synth.C5_P, synth.C5_Q, synth.C5_OMEGA_SEED
    mats, a64 = [], []
    for b, (m, n) in enumerate(shapes):
        a, *_ = synth.c5_matrix(b)
        ab = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16)
        t = torch.zeros(m, -(-n // 8) * 8, dtype=torch.bfloat16, device="cuda")
        t[:, :n] = ab.cuda()
        mats.append(t)
        a64.append(ab.double().numpy())
    with pkg.BatchedPlan(shapes, k, p, q, seed=seed) as pl:
        pl.svd(mats)
        grads = pl.backward(mats)
        pl.sync()
    rng = np.random.default_rng(8)
    worst = 0.0
    for b, (m, n) in enumerate(shapes):
        om = torch.tensor(philox.gaussian(seed + b, 0, n, k + p), dtype=torch.float32)
        om = om.to(torch.bfloat16).double().numpy()
        dirs = []
        for _ in range(4):
            e = rng.standard_normal((m, n))
            dirs.append(e / np.linalg.norm(e))
        fd = grad.grad_fd(a64[b], k, p, q, om, h=1e-3, directions=dirs)
        g = _np(grads[b])
        ad = np.array([np.sum(g * e) for e in dirs])
        err = np.abs(ad - fd) / (np.abs(fd) + 1e-3 * np.linalg.norm(g))
        worst = max(worst, float(err.max()))
        print(f"C5 matrix {b} ({m}x{n}): directional derivatives {ad} vs FD {fd}")
        assert np.all(err <= 1e-3), err
    print(f"C5 first 8: worst relative directional error {worst:.3e}")
