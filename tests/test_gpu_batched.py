"""GPU parity of the batched randomized SVD (many small bfloat16 matrices, one plan).

Each matrix b is checked against the oracle run on the same bfloat16 values with its
own test matrix Omega_b = gaussian(seed + b, stream 0): singular values within
eps sigma_1 + 2 (the oracle's own shortfall from the true singular values), never
above the true singular values, vectors within the Wedin gap bound -- the same
acceptance as the single-matrix tensor-core path (tests/test_gpu_tc.py, _check_ritz).
"""
import os
import sys

import numpy as np
import pytest
import torch

import synth
from oracle import philox

sys.path.insert(0, os.path.dirname(__file__))
from test_gpu_tc import _check_ritz  # noqa: E402

pytestmark = pytest.mark.gpu

SHAPES = [(300, 200), (128, 64), (517, 389), (1000, 777), (2048, 1024), (129, 65), (640, 130),
          (1500, 64)]


def _make_batch(shapes, seed):
    mats, a64 = [], []
    for b, (m, n) in enumerate(shapes):
        sig = np.exp(-np.arange(min(m, n)) / 4.0)
        a, *_ = synth.lowrank(m, n, sig, seed + b)
        ab = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16)
        lda = -(-n // 8) * 8
        t = torch.zeros(m, lda, dtype=torch.bfloat16, device="cuda")
        t[:, :n] = ab.cuda()
        mats.append(t)
        a64.append(ab.float().numpy().astype(np.float64))
    return mats, a64


@pytest.mark.parametrize("k,p,q", [(16, 8, 1), (10, 6, 0), (8, 8, 2)])
def test_batched_rsvd_matches_oracle(rsvd_lib, k, p, q):
    seed = 2005
    mats, a64 = _make_batch(SHAPES, 1005)
    with rsvd_lib.BatchedPlan(SHAPES, k, p, q, seed=seed) as pl:
        U, S, V = pl.svd(mats)
        sweeps = pl.sync()
        u_all, s_all, v_all = U.cpu().double().numpy(), S.cpu().double().numpy(), V.cpu().double().numpy()
        rm, rn = pl.row_m, pl.row_n
    assert 0 < sweeps < 40
    for b, (m, n) in enumerate(SHAPES):
        om = philox.gaussian(seed + b, 0, n, k + p)
        _check_ritz(a64[b], u_all[rm[b]:rm[b + 1]], s_all[b], v_all[rn[b]:rn[b + 1]], k, p, q, om)


def test_batched_matches_single_matrix_path(rsvd_lib):
    """The batched plan and the one-matrix plan agree on a matrix they both accept."""
    m, n, k, p, q = 700, 512, 16, 8, 1
    mats, a64 = _make_batch([(m, n)], 77)
    with rsvd_lib.BatchedPlan([(m, n)], k, p, q, seed=9) as pl:
        U, S, V = pl.svd(mats)
        pl.sync()
    with rsvd_lib.Plan(m, n, k, p, q, 9, rsvd_lib.RSVD_BF16_TC) as sp:
        U1, S1, V1 = sp.svd(mats[0][:, :n].contiguous())
        torch.cuda.synchronize()
    s, s1 = S[0].cpu().double().numpy(), S1.cpu().double().numpy()
    assert np.max(np.abs(s - s1)) <= 1e-4 * s1[0]


def _omega_bf16(pkg, seed, n, l):
    om = torch.zeros(n, l, device="cuda")
    pkg.rsvd_draw_gaussian(seed, 0, n, l, om, l)
    torch.cuda.synchronize()
    return om.to(torch.bfloat16).double().cpu().numpy()


@pytest.mark.parametrize("q", [1, 0])
def test_batched_backward_matches_autograd(rsvd_lib, q):
    """dL/dA_b from the library against torch autograd through the oracle's float64 steps
    (Householder QR with the sign fix, SVD of B), on the same bfloat16 A_b and the
    bfloat16 test matrix the first pass multiplies with.  The terms 2 A + U (I - 2S) V^T
    are float32-accurate; the chain terms (through the range finder) pass through
    R_0^-T, so float32 rounding in them is amplified by kappa(Y_0) = kappa(R_0):
        ||dA - dA_ref||_F / ||dA_ref||_F <= 1e-4 + 20 u32 kappa(Y_0) c,
    c = the chain terms' share of ||dA_ref||_F (measured against the closed form
    2 (A - A_k) + U_k V_k^T of the exact truncated SVD)."""
    from oracle import grad

    shapes = [(300, 200), (128, 64), (517, 389), (700, 512)]
    k, p, seed = 16, 8, 7
    mats, a64 = _make_batch(shapes, 1105)
    with rsvd_lib.BatchedPlan(shapes, k, p, q, seed=seed) as pl:
        pl.svd(mats)
        grads = pl.backward(mats)
        pl.sync()
    for b, (m, n) in enumerate(shapes):
        om = _omega_bf16(rsvd_lib, seed + b, n, k + p)
        g_ref = grad.grad_autograd(a64[b], k, p, q, om)
        g = grads[b].double().cpu().numpy()
        rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
        chain = np.linalg.norm(g_ref - grad.grad_exact_svd(a64[b], k)) / np.linalg.norm(g_ref)
        kap = np.linalg.cond(a64[b] @ om)
        tol = 1e-4 + 20 * 2.0 ** -24 * kap * chain
        print(f"backward b={b} q={q}: rel err {rel:.3e}  chain share {chain:.3e}  kappa(Y0) {kap:.3e}  tol {tol:.3e}")
        assert rel <= tol, (rel, tol)


def test_batched_graph_replay_and_autotuner(rsvd_lib, tmp_path, monkeypatch):
    """The first call times the grouped pass's configurations (autotuner, cached in the JSON
    file named by RSVD_TUNE_CACHE) and captures the forward in a CUDA graph; later calls
    replay it.  Replays give the same bits; a second plan of the same shape class reads
    the cache instead of timing."""
    import json

    cache = tmp_path / "tune.json"
    monkeypatch.setenv("RSVD_TUNE_CACHE", str(cache))
    shapes = SHAPES[:5]
    mats, _ = _make_batch(shapes, 1205)
    with rsvd_lib.BatchedPlan(shapes, 16, 8, 1, seed=5) as pl:
        U1, S1, V1 = pl.svd(mats)
        U2, S2, V2 = pl.svd(mats, *[torch.empty_like(t) for t in (U1, S1, V1)])
        t = pl.tuning()
        g1 = pl.backward(mats)
        g2 = pl.backward(mats)
        pl.sync()
    assert t["tuned"] and all(2 <= s <= 8 for s in t["stages"]) and all(c in (1, 2) for c in t["ctas_per_sm"])
    assert torch.equal(U1, U2) and torch.equal(S1, S2) and torch.equal(V1, V2)
    assert all(torch.equal(a, b) for a, b in zip(g1, g2))
    entries = json.loads(cache.read_text())
    assert len(entries) == 1 and len(next(iter(entries.values()))) == 8
    with rsvd_lib.BatchedPlan(shapes, 16, 8, 1, seed=5) as pl2:
        pl2.svd(mats)
        assert pl2.tuning() == t
        pl2.sync()


def test_batched_full_c5_batch(rsvd_lib):
    """The timed batched configuration itself: 512 matrices of the C5 shapes (m ~ U[128, 2048],
    n ~ U[64, 1024]), k = 16, p = 8, q = 1, built on the device as the bench builds them.
    Sixteen matrices (the first eight and eight spread over the batch) are checked against
    the oracle: the forward with the acceptance of the tests above, the backward against
    autograd through the oracle's float64 steps with the same tolerance rule."""
    from oracle import grad

    pkg = rsvd_lib
    shapes = synth.c5_shapes()
    k, p, q, seed = synth.C5_K, synth.C5_P, synth.C5_Q, synth.C5_OMEGA_SEED
    mats = []
    for b, (m, n) in enumerate(shapes):
        a = synth.device_lowrank(m, n, synth.spectrum_exp(min(m, n), 4.0), synth.C5_MATRIX_SEED * 100003 + b)
        t = torch.zeros(m, -(-n // 8) * 8, dtype=torch.bfloat16, device="cuda")
        t[:, :n] = a.to(torch.bfloat16)
        mats.append(t)
    with pkg.BatchedPlan(shapes, k, p, q, seed=seed) as pl:
        U, S, V = pl.svd(mats)
        grads = pl.backward(mats)
        sweeps = pl.sync()
        u_all, s_all, v_all = U.cpu().double().numpy(), S.cpu().double().numpy(), V.cpu().double().numpy()
        rm, rn = pl.row_m, pl.row_n
    assert 0 < sweeps < 40
    picks = list(range(8)) + list(range(40, len(shapes), (len(shapes) - 40) // 8))[:8]
    for b in picks:
        m, n = shapes[b]
        a64 = mats[b][:, :n].double().cpu().numpy()
        om = philox.gaussian(seed + b, 0, n, k + p)
        _check_ritz(a64, u_all[rm[b]:rm[b + 1]], s_all[b], v_all[rn[b]:rn[b + 1]], k, p, q, om)
        omb = _omega_bf16(pkg, seed + b, n, k + p)
        g_ref = grad.grad_autograd(a64, k, p, q, omb)
        g = grads[b].double().cpu().numpy()
        rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
        chain = np.linalg.norm(g_ref - grad.grad_exact_svd(a64, k)) / np.linalg.norm(g_ref)
        tol = 1e-4 + 20 * 2.0 ** -24 * np.linalg.cond(a64 @ omb) * chain
        assert rel <= tol, (b, rel, tol)
