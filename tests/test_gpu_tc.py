"""GPU parity of the bfloat16 tensor-core path (tcgen05) against the float64 oracle.

A pass over A multiplies bfloat16 A by the bfloat16-rounded operand with
float32 accumulation; products of two bfloat16 numbers are exact in float32,
so against the float64 product of the same bfloat16 inputs the only error is
the float32 accumulation: |Y - Y_ref| <= 1e-5 (|A| |X|)_ij.

End to end, the tensor-core path rounds the test matrix and the intermediate
bases to bfloat16 (relative 2^-9), which changes the sampled subspace a
little; the singular values it returns are Ritz values of A on that subspace.
Against the oracle run on the same bfloat16 A with the same Omega (float64),
both sets are Ritz values of nearly the same quality: the difference is
bounded by the oracle's own shortfall sigma_i(A) - sigma_i_ref (a Ritz value
moves second-order in the subspace angle) plus the float32 target 1e-5
sigma_1.  The final pass uses a hi + lo split of the basis, so B = Q^T A is
float32-accurate for the bfloat16 A.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import metrics, mixed, philox, rsvd64

pytestmark = pytest.mark.gpu


def _dev(x, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def _np(t):
    return t.detach().float().cpu().numpy().astype(np.float64)


def _bf16(x):
    return synth.bf16_round(x)


def _plan(pkg, m, n, k, p, q, seed, lda=0, rounds=3):
    return pkg.Plan(m, n, k, p, q, seed, pkg.RSVD_BF16_TC, rounds, lda=lda)


@pytest.mark.parametrize("m,n,l,lda", [(512, 384, 32, 0), (517, 1000, 16, 0), (1000, 520, 112, 0),
                                       (300, 389, 48, 392), (2048, 4096, 128, 0), (700, 640, 160, 0),
                                       (1000, 1104, 256, 0)])
def test_tc_sketch_matches_oracle(rsvd_lib, m, n, l, lda):
    rng = np.random.default_rng(m * 3 + n)
    ld = lda if lda else n
    a = _bf16(rng.standard_normal((m, n)))
    a_store = np.zeros((m, ld))
    a_store[:, :n] = a
    A = _dev(a_store, torch.bfloat16)
    with _plan(rsvd_lib, m, n, l, 0, 0, 1, lda=ld) as pl:
        for trans in (0, 1):
            kx = m if trans else n
            x = philox.gaussian(5 + trans, 0, kx, l).astype(np.float32)
            Y = torch.zeros((n if trans else m), l, device="cuda")
            rsvd_lib.rsvd_sketch(pl.handle, A, trans, _dev(x), Y)
            assert rsvd_lib.rsvd_sync(pl.handle) == rsvd_lib.RSVD_OK
            xb = _bf16(x)
            op = a.T if trans else a
            ref = op @ xb
            bound = 1e-5 * (np.abs(op) @ np.abs(xb)) + 1e-30
            err = np.abs(_np(Y) - ref)
            assert np.all(err <= bound), (trans, (err / bound).max())


def _tc_svd(pkg, a_bf, k, p, q, seed):
    m, n = a_bf.shape
    with _plan(pkg, m, n, k, p, q, seed) as pl:
        U, S, V = pl.svd(_dev(a_bf, torch.bfloat16))
    return _np(U), _np(S), _np(V)


def _check_ritz(a64, u, s, v, k, p, q, omega, eps=1e-5, vec_eps=None):
    uf, sf, vf, _ = rsvd64.rsvd(a64, k + p, 0, q, omega)
    sr = sf[:k]
    s_true = np.linalg.svd(a64, compute_uv=False)[:k] if a64.size <= 4e6 else sr
    shortfall = np.maximum(s_true - sr, 0.0)
    tol = eps * sr[0] + 2.0 * shortfall
    assert np.all(np.abs(s - sr) <= tol), (np.abs(s - sr) / tol).max()
    assert np.all(s <= s_true * (1 + 1e-5) + 1e-6 * sr[0])          # Ritz values never exceed sigma_i
    bound = metrics.gap_bound(sr, vec_eps or eps, c=1.0, s_next=sf[k]) + np.sqrt(2.0 * shortfall / sr)
    d = np.sign(np.sum(u * uf[:, :k], axis=0))
    d[d == 0] = 1
    assert np.all(np.linalg.norm(u * d - uf[:, :k], axis=0) <= bound + 1e-4)
    assert np.all(np.linalg.norm(v * d - vf[:, :k], axis=0) <= bound + 1e-4)
    assert metrics.orthonormality(u) <= 2e-5 and metrics.orthonormality(v) <= 2e-5


def test_tc_rsvd_c1_full_size(rsvd_lib):
    w = synth.C1
    a, *_ = synth.lowrank(w.m, w.n, w.sigma(), w.matrix_seed)
    ab = _bf16(a)
    u, s, v = _tc_svd(rsvd_lib, ab, w.k, w.p, w.q, w.omega_seed)
    om = philox.gaussian(w.omega_seed, 0, w.n, w.l)
    _check_ritz(ab, u, s, v, w.k, w.p, w.q, om)


# l_p = 160, 208 and 256 take the tensor-core Gram and apply of the orthonormaliser (l_p > 128),
# with the one-CTA (160) and the row-packed (208, 256) factorisation (n a multiple of 8: the
# bfloat16 rows of A must start on 16-byte boundaries)
@pytest.mark.parametrize("m,n,k,p,q", [(1024, 768, 30, 10, 1), (777, 520, 12, 4, 2), (3000, 256, 100, 12, 1),
                                       (1104, 896, 236, 20, 1), (1501, 704, 150, 10, 1),
                                       (903, 1304, 190, 18, 2)])
def test_tc_rsvd_shapes(rsvd_lib, m, n, k, p, q):
    a, *_ = synth.lowrank(m, n, synth.spectrum_exp(min(m, n), 9.0), m + n)
    ab = _bf16(a)
    u, s, v = _tc_svd(rsvd_lib, ab, k, p, q, 3)
    om = philox.gaussian(3, 0, n, k + p)
    _check_ritz(ab, u, s, v, k, p, q, om)


def test_tc_matched_error_against_fp32_c1(rsvd_lib):
    """Reconstruction error of the tensor-core path on the bfloat16 copy, measured
    against the float32 matrix, exceeds the plain FP32 path's by a small fraction."""
    w = synth.C1
    a, *_ = synth.lowrank(w.m, w.n, w.sigma(), w.matrix_seed)
    a32 = a.astype(np.float32)
    with rsvd_lib.Plan(w.m, w.n, w.k, w.p, w.q, w.omega_seed) as pl:
        U, S, V = pl.svd(_dev(a32))
    e32 = metrics.fro_error(a32.astype(np.float64), _np(U), _np(S), _np(V))
    u, s, v = _tc_svd(rsvd_lib, _bf16(a32), w.k, w.p, w.q, w.omega_seed)
    etc = metrics.fro_error(a32.astype(np.float64), u, s, v)
    assert (etc - e32) / e32 <= 1e-4, (etc - e32) / e32


def test_convert_a_hi_lo_exact(rsvd_lib):
    rng = np.random.default_rng(2)
    a = rng.standard_normal((300, 261)).astype(np.float32) * np.float32(3.7)
    out = torch.zeros(600, 264, dtype=torch.bfloat16, device="cuda")
    rsvd_lib.rsvd_convert_a(_dev(a), 300, 261, 261, out, 264, 1)
    torch.cuda.synchronize()
    o = out.float().cpu().numpy().astype(np.float64)
    hi = _bf16(a)
    lo = _bf16(a.astype(np.float64) - hi)
    assert np.array_equal(o[:300, :261], hi) and np.array_equal(o[300:, :261], lo)
    # hi + lo carries ~16 significant bits of A
    assert np.max(np.abs(hi + lo - a) / np.abs(a)) <= 2.0 ** -16


def _tc_svd_hilo(pkg, a32, k, p, q, seed):
    m, n = a32.shape
    A = _dev(a32)
    with pkg.Plan(m, n, k, p, q, seed, pkg.RSVD_BF16_TC, dtype=pkg.RSVD_BF16X2) as pl:
        U, S, V = pl.svd(pkg.split_bf16(A))
    return _np(U), _np(S), _np(V)


def test_tc_hilo_rsvd_c1_full_size(rsvd_lib):
    """Residual-corrected final pass: B = Q^T A from hi + lo, checked against the oracle
    on the float32 A (Ritz tolerance as above plus the bfloat16 subspace of Stage A)."""
    w = synth.C1
    a, *_ = synth.lowrank(w.m, w.n, w.sigma(), w.matrix_seed)
    a32 = a.astype(np.float32)
    u, s, v = _tc_svd_hilo(rsvd_lib, a32, w.k, w.p, w.q, w.omega_seed)
    om = philox.gaussian(w.omega_seed, 0, w.n, w.l)
    # Stage A sampled bf16(A): its subspace, and so U and V, differ from the oracle's on A by
    # up to ||A - bf16(A)||_2 / gap (Wedin); B itself sees A through hi + lo
    a64 = a32.astype(np.float64)
    e_rel = np.linalg.norm(a64 - _bf16(a32), 2) / w.sigma()[0]
    _check_ritz(a64, u, s, v, w.k, w.p, w.q, om, vec_eps=max(1e-5, e_rel))


def test_tc_hilo_matched_error_c1(rsvd_lib):
    w = synth.C1
    a, *_ = synth.lowrank(w.m, w.n, w.sigma(), w.matrix_seed)
    a32 = a.astype(np.float32)
    with rsvd_lib.Plan(w.m, w.n, w.k, w.p, w.q, w.omega_seed) as pl:
        U, S, V = pl.svd(_dev(a32))
    e32 = metrics.fro_error(a32.astype(np.float64), _np(U), _np(S), _np(V))
    u, s, v = _tc_svd_hilo(rsvd_lib, a32, w.k, w.p, w.q, w.omega_seed)
    etc = metrics.fro_error(a32.astype(np.float64), u, s, v)
    assert abs(etc - e32) / e32 <= 1e-4, (etc - e32) / e32


@pytest.mark.parametrize("m,n,l", [(1000, 520, 112), (517, 1000, 48), (700, 640, 160)])
def test_tc_sketch_with_residual_matches_oracle(rsvd_lib, m, n, l):
    """Every pass reading hi + lo (residual_passes = 1): Y = (hi + lo) bf16(X) and
    Y = (hi + lo)^T bf16(X), against the float64 product of the same operands."""
    rng = np.random.default_rng(m + 7 * n)
    a = (rng.standard_normal((m, n)) * 3.1).astype(np.float32)
    A = rsvd_lib.split_bf16(_dev(a))
    hi = _bf16(a)
    hl = hi + _bf16(a.astype(np.float64) - hi)
    with rsvd_lib.Plan(m, n, l, 0, 0, 1, rsvd_lib.RSVD_BF16_TC, dtype=rsvd_lib.RSVD_BF16X2,
                       residual_passes=1) as pl:
        for trans in (0, 1):
            kx = m if trans else n
            x = philox.gaussian(9 + trans, 0, kx, l).astype(np.float32)
            Y = torch.zeros((n if trans else m), l, device="cuda")
            rsvd_lib.rsvd_sketch(pl.handle, A, trans, _dev(x), Y)
            assert rsvd_lib.rsvd_sync(pl.handle) == rsvd_lib.RSVD_OK
            xb = _bf16(x)
            op = hl.T if trans else hl
            ref = op @ xb
            bound = 1e-5 * (np.abs(op) @ np.abs(xb)) + 1e-30
            err = np.abs(_np(Y) - ref)
            assert np.all(err <= bound), (trans, (err / bound).max())


def test_tc_residual_every_pass_matched_error(rsvd_lib):
    """A slow-decay 3072 x 3072 matrix (sigma_j = j^-1.5, k = 100, p = 10, q = 1): with only
    the final pass reading the residual, the bfloat16 subspace of Stage A moves the
    reconstruction error by a few 1e-4 relative; with every pass reading hi + lo the error
    matches the float32 path's to 1e-4."""
    m = n = 3072
    k, p, q, seed = 100, 10, 1, 11
    a, *_ = synth.lowrank(m, n, np.arange(1, n + 1, dtype=np.float64) ** -1.5, 4242)
    a32 = a.astype(np.float32)
    with rsvd_lib.Plan(m, n, k, p, q, seed) as pl:
        U, S, V = pl.svd(_dev(a32))
    e32 = metrics.fro_error(a32.astype(np.float64), _np(U), _np(S), _np(V))
    with rsvd_lib.Plan(m, n, k, p, q, seed, rsvd_lib.RSVD_BF16_TC, dtype=rsvd_lib.RSVD_BF16X2,
                       residual_passes=1) as pl:
        U, S, V = pl.svd(rsvd_lib.split_bf16(_dev(a32)))
    etc = metrics.fro_error(a32.astype(np.float64), _np(U), _np(S), _np(V))
    assert abs(etc - e32) / e32 <= 1e-4, (etc - e32) / e32


def test_tc_residual_final_bases_matches_oracle(rsvd_lib):
    """residual_passes = 2 (the residual lo read by the last pass of Stage A and by the final
    pass, hi alone by the earlier one) on a 2048 x 2048 slow-decay matrix (sigma_j = j^-1.5,
    k = 100, p = 10, q = 1), against oracle.mixed with the same pattern and the same Omega:
    sigma within 1e-5 sigma_1 and the singular vectors within Wedin's bound for a 1e-5
    sigma_1 perturbation (the float32 targets)."""
    m = n = 2048
    k, p, q, seed = 100, 10, 1, 5
    l = k + p
    a, *_ = synth.lowrank(m, n, np.arange(1, n + 1, dtype=np.float64) ** -1.5, 4343)
    a32 = a.astype(np.float32)
    with rsvd_lib.Plan(m, n, k, p, q, seed, rsvd_lib.RSVD_BF16_TC, dtype=rsvd_lib.RSVD_BF16X2,
                       residual_passes=2) as pl:
        U, S, V = pl.svd(rsvd_lib.split_bf16(_dev(a32)))
        assert rsvd_lib.rsvd_sync(pl.handle) == rsvd_lib.RSVD_OK
    u, s, v = _np(U), _np(S), _np(V)
    hi = _bf16(a32)
    hl = hi + _bf16(a32.astype(np.float64) - hi)
    om = philox.gaussian(seed, philox.STREAM_OMEGA, n, l)
    um, sm, vm, _ = mixed.rsvd(hi, l, 0, q, om, a_final=hl, a_last=hl)
    sr = sm[:k]
    assert np.max(np.abs(s - sr)) <= 1e-5 * sr[0], np.max(np.abs(s - sr)) / sr[0]
    bound = metrics.gap_bound(sr, 1e-5, c=1.0, s_next=sm[k]) + 1e-5
    for x, xr in ((u, um[:, :k]), (v, vm[:, :k])):
        d = np.sign(np.sum(x * xr, axis=0))
        d[d == 0] = 1.0
        dist = np.linalg.norm(x * d - xr, axis=0)
        assert np.all(dist <= bound), (dist / bound).max()
