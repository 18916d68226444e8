"""GPU parity of the single-pass randomized SVD (Section 5.5) against the oracle.

Both sides take the same Omega (Gaussian, stream 0, n x l) and Psi (Gaussian, stream 1,
m x l' with the library's default l' = min(3 l, 256, n)): the library's own draws, read
back through the C ABI, feed the oracle.  B is the
minimum-residual solution of B X1 = C1, B^T X2 = C2 through the Sylvester normal
equations; its float32 error grows with the conditioning of that system.  A
first-order bound: a relative perturbation u of the inputs moves B by about
u (kappa(X1)^2 + kappa(X2)^2) ||B|| (the normal equations square the conditioning
of each side), so singular values are compared within
    tol = 2 u32 (kappa(X1)^2 + kappa(X2)^2) sigma_1,     u32 = 2^-24,
and the singular subspaces through the Wedin gap bound at that tolerance.  (Measured
errors sit 10-30x below it: 0.7e-5 to 4.6e-5 sigma_1 at kappa^2 sums near 1e4.)
Exact-rank inputs (rank r < k) must come back exactly up to the same tolerance, with
the trailing singular values at that level too.
"""
import os
import sys

import numpy as np
import pytest
import torch

import synth
from oracle import metrics, single_pass

sys.path.insert(0, os.path.dirname(__file__))
from test_gpu_parity import _dev, _np  # noqa: E402

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def psi_cols(m, n, l):
    """The library's default width l' of Psi: min(3 l, 256, n)."""
    return min(3 * l, 256, n)


def _draws(pkg, pl, m, n, l, seed, bf16):
    om = torch.zeros(n, l, device="cuda")
    pkg.rsvd_get_omega(pl.handle, om)
    lt = psi_cols(m, n, l)
    psi = torch.zeros(m, lt, device="cuda")
    pkg.rsvd_draw_gaussian(seed, 1, m, lt, psi, lt)
    torch.cuda.synchronize()
    if bf16:
        om, psi = om.to(torch.bfloat16).float(), psi.to(torch.bfloat16).float()
    return _np(om), _np(psi)


def _run(pkg, a, k, p, seed, precision):
    m, n = a.shape
    l = k + p
    bf16 = precision == pkg.RSVD_BF16_TC
    with pkg.Plan(m, n, k, p, 0, seed, precision, single_pass=1) as pl:
        om, psi = _draws(pkg, pl, m, n, l, seed, bf16)
        A = _dev(a, torch.bfloat16 if bf16 else torch.float32)
        U, S, V = pl.svd(A)
        torch.cuda.synchronize()
        bits, _ = pkg.rsvd_diagnostics(pl.handle)
    return _np(U), _np(S), _np(V), om, psi, bits


def _oracle(a64, k, om, psi):
    u, s, v, (qm, qt, b) = single_pass.rsvd_single_pass(a64, k, om, psi)
    y, yt = single_pass.two_sided_sketch(a64, om, psi)
    x1, _, x2, _ = single_pass.reduced_system(qm, qt, om, psi, y, yt)
    kap = np.linalg.cond(x1) ** 2 + np.linalg.cond(x2) ** 2
    sb = np.linalg.svd(b, compute_uv=False)
    return u, s, v, sb, kap


def _compare(u, s, v, ur, sr, vr, sb_full, k, tol):
    assert np.max(np.abs(s - sr)) <= tol, (np.max(np.abs(s - sr)), tol)
    eps = tol / sr[0]
    bound = metrics.gap_bound(sr, eps, s_next=sb_full[k] if k < len(sb_full) else None)
    d = np.sign(np.sum(u * ur, axis=0))
    d[d == 0] = 1
    du = np.linalg.norm(u * d - ur, axis=0)
    dv = np.linalg.norm(v * d - vr, axis=0)
    print("  vectors: max du", du.max(), "max dv", dv.max(), "min bound", (bound + 1e-5).min(),
          "worst ratio", max((du / (bound + 1e-5)).max(), (dv / (bound + 1e-5)).max()))
    assert np.all(du <= bound + 1e-5)
    assert np.all(dv <= bound + 1e-5)
    assert metrics.orthonormality(u) <= 1e-5 and metrics.orthonormality(v) <= 1e-5


@pytest.mark.parametrize("m,n,k,p", [(4096, 512, 16, 8), (2000, 700, 30, 10), (517, 1031, 12, 6)])
def test_single_pass_fp32_matches_oracle(rsvd_lib, m, n, k, p):
    sig = synth.spectrum_exp(min(m, n), 20.0)
    a, *_ = synth.lowrank(m, n, sig, 7 * m + n)
    a32 = a.astype(np.float32)
    u, s, v, om, psi, bits = _run(rsvd_lib, a32, k, p, 41, rsvd_lib.RSVD_PLAIN_FP32)
    assert not bits & 3
    ur, sr, vr, sb, kap = _oracle(a32.astype(np.float64), k, om, psi)
    tol = 2 * U32 * kap * sr[0]
    print("single pass fp32: max dsigma/sigma1", np.max(np.abs(s - sr)) / sr[0], "tol/sigma1", tol / sr[0])
    _compare(u, s, v, ur, sr, vr, sb, k, tol)


def test_single_pass_bf16_tc_matches_oracle(rsvd_lib):
    m, n, k, p = 4096, 512, 16, 8
    sig = synth.spectrum_exp(n, 20.0)
    a, *_ = synth.lowrank(m, n, sig, 99)
    ab = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).float().numpy()
    u, s, v, om, psi, bits = _run(rsvd_lib, ab, k, p, 43, rsvd_lib.RSVD_BF16_TC)
    ur, sr, vr, sb, kap = _oracle(ab.astype(np.float64), k, om, psi)
    tol = 2 * U32 * kap * sr[0]
    print("single pass bf16: max dsigma/sigma1", np.max(np.abs(s - sr)) / sr[0], "tol/sigma1", tol / sr[0])
    _compare(u, s, v, ur, sr, vr, sb, k, tol)


def test_single_pass_exact_rank(rsvd_lib):
    """rank r < k: the two sketches capture A exactly, so B reproduces its spectrum."""
    m, n, r, k, p = 3000, 400, 6, 10, 6
    sig = np.zeros(n)
    sig[:r] = np.linspace(1.0, 0.3, r)
    a, *_ = synth.lowrank(m, n, sig, 5)
    a32 = a.astype(np.float32)
    u, s, v, om, psi, bits = _run(rsvd_lib, a32, k, p, 3, 0)
    st = np.linalg.svd(a32.astype(np.float64), compute_uv=False)
    *_, kap = _oracle(a32.astype(np.float64), k, om, psi)
    tol = 2 * U32 * kap * st[0]
    print("single pass exact rank: max dsigma/sigma1", np.max(np.abs(s[:r] - st[:r])) / st[0], "tol/sigma1", tol / st[0])
    assert np.max(np.abs(s[:r] - st[:r])) <= tol
    assert np.max(np.abs(s[r:])) <= tol


@pytest.mark.parametrize("precision", [0, 1])
def test_single_pass_noisy_tall_workload(rsvd_lib, precision):
    """The tall-skinny workload's recipe at 16384 x 1024 (sigma_j = max(e^-(j-1)/20, 1e-6),
    k = 64, p = 16, iid Gaussian noise scaled so that its Frobenius norm equals that of the
    signal, as the 262144 x 4096 workload's does): the relative reconstruction error
    ||A - U S V^T||_F / ||A||_F of the GPU stays within 2 % of the oracle's on the same
    Omega and Psi, and below 1 (the error of the zero approximation)."""
    pkg = rsvd_lib
    m, n, k, p, seed = 16384, 1024, 64, 16, 47
    sig = synth.spectrum_exp_floor(n, 20.0, 1e-6)
    a, *_ = synth.lowrank(m, n, sig, 1003)
    a += synth.noise(m, n, float(np.sqrt(np.sum(sig ** 2) / (m * n))), 77)
    a32 = a.astype(np.float32)
    if precision == pkg.RSVD_BF16_TC:
        a32 = torch.tensor(a32).to(torch.bfloat16).float().numpy()
    a64 = a32.astype(np.float64)
    u, s, v, om, psi, bits = _run(pkg, a32, k, p, seed, precision)
    ur, sr, vr, _, kap = _oracle(a64, k, om, psi)
    nrm = np.linalg.norm(a64)
    e_gpu = np.linalg.norm(a64 - (u * s) @ v.T) / nrm
    e_ref = np.linalg.norm(a64 - (ur * sr) @ vr.T) / nrm
    print(f"noisy tall single pass (precision {precision}): GPU {e_gpu:.5f} oracle {e_ref:.5f} "
          f"max dsigma/sigma1 {np.max(np.abs(s - sr)) / sr[0]:.2e}")
    assert e_gpu <= 1.02 * e_ref and e_gpu < 1.0
    assert np.max(np.abs(s - sr)) <= 2 * U32 * kap * sr[0]


@pytest.mark.parametrize("precision", [0, 1])
def test_single_pass_repeated_calls_agree(rsvd_lib, precision):
    """Psi is drawn by a plan's first single pass and kept: a second and third call on the
    same plan (with other passes' operands written in between) give the same factors bit
    for bit."""
    pkg = rsvd_lib
    m, n, k, p = 3000, 1024, 40, 8
    rng = np.random.default_rng(4)
    a = (rng.standard_normal((m, 60)) @ rng.standard_normal((60, n))).astype(np.float32)
    bf16 = precision == pkg.RSVD_BF16_TC
    A = torch.tensor(a, device="cuda", dtype=torch.bfloat16 if bf16 else torch.float32)
    with pkg.Plan(m, n, k, p, 0, 9, precision, single_pass=1) as pl:
        outs = []
        for _ in range(3):
            U, S, V = pl.svd(A)
            torch.cuda.synchronize()
            outs.append((U.clone(), S.clone(), V.clone()))
    for U, S, V in outs[1:]:
        assert torch.equal(U, outs[0][0]) and torch.equal(S, outs[0][1]) and torch.equal(V, outs[0][2])
