"""GPU parity of the C-ABI library against the float64 oracle (plain FP32 path).

Every call goes through the C ABI (paper_0909_4061_gb300 is argument marshalling
only).  Tolerances:
  * test matrix: the integer part of the generator is shared exactly; the
    float32 Box-Muller differs from the float64 one by a few ulp:
    |z_gpu - z_ref| <= 4e-6 max(1, |z|);
  * one pass over A: float32 accumulation over K terms,
    |Y_gpu - Y_ref| <= 1e-5 (|A| |X|)_ij;
  * singular values: |sigma_gpu - sigma_ref| <= 1e-5 sigma_1 (the stated
    float32 target);
  * singular vectors, compared after a per-column sign alignment: a
    perturbation of size 1e-5 sigma_1 turns u_j by at most about
    1e-5 sigma_1 / gap_j (Wedin), gap_j the distance of sigma_j to its
    neighbours (sigma_{k+1} for the last one);
  * orthonormal bases: max |Q^T Q - I| <= 1e-5.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import jacobi as ojacobi
from oracle import metrics, philox, rsvd64

pytestmark = pytest.mark.gpu

EPS_SIGMA = 1e-5


def _dev(x, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def _np(t):
    return t.detach().float().cpu().numpy().astype(np.float64)


def _gpu_svd(pkg, a32, k, p, q, seed, precision=0, rounds=3, omega=None):
    m, n = a32.shape
    with pkg.Plan(m, n, k, p, q, seed, precision, rounds) as pl:
        if omega is not None:
            om = _dev(omega)
            pkg.rsvd_set_omega(pl.handle, om)
        A = _dev(a32, torch.bfloat16 if precision == pkg.RSVD_BF16_TC else torch.float32)
        U, S, V = pl.svd(A)
        torch.cuda.synchronize()
        return _np(U), _np(S), _np(V)


def _check_svd(a64, u, s, v, k, p, q, omega, eps=EPS_SIGMA, vec_c=1.0):
    uf, sf, vf, _ = rsvd64.rsvd(a64, k + p, 0, q, omega)      # untruncated: sigma_{k+1} too
    ur, sr, vr = uf[:, :k], sf[:k], vf[:, :k]
    assert np.max(np.abs(s - sr)) <= eps * sr[0], np.max(np.abs(s - sr)) / sr[0]
    bound = metrics.gap_bound(sr, eps, c=vec_c, s_next=sf[k] if k < len(sf) else None)
    # align each pair (u_j, v_j) by the sign of u_j . u_j_ref
    d = np.sign(np.sum(u * ur, axis=0))
    d[d == 0] = 1
    du = np.linalg.norm(u * d - ur, axis=0)
    dv = np.linalg.norm(v * d - vr, axis=0)
    assert np.all(du <= bound + 1e-5), (du / (bound + 1e-5)).max()
    assert np.all(dv <= bound + 1e-5), (dv / (bound + 1e-5)).max()
    return sr


# --------------------------------------------------------------------------
# step a1: the test matrix
# --------------------------------------------------------------------------


@pytest.mark.parametrize("rows,cols,seed,stream", [(1, 1, 0, 0), (7, 5, 3, 0), (1000, 30, 2001, 0),
                                                   (33, 257, 12345678901, 1), (4096, 80, 9, 1)])
def test_draw_gaussian_matches_oracle(rsvd_lib, rows, cols, seed, stream):
    out = torch.full((rows, cols + 3), 7.0, device="cuda")
    rsvd_lib.rsvd_draw_gaussian(seed, stream, rows, cols, out, cols + 3)
    torch.cuda.synchronize()
    z = _np(out)
    ref = philox.gaussian(seed, stream, rows, cols)
    assert np.all(np.abs(z[:, :cols] - ref) <= 4e-6 * np.maximum(1.0, np.abs(ref)))
    assert np.all(z[:, cols:] == 7.0)          # nothing written past cols


# --------------------------------------------------------------------------
# steps a2/a4/a5: one pass over A
# --------------------------------------------------------------------------


@pytest.mark.parametrize("m,n,l", [(517, 389, 32), (389, 517, 17), (2000, 1000, 30)])
def test_sketch_fp32_matches_oracle(rsvd_lib, m, n, l):
    rng = np.random.default_rng(m + n)
    a = rng.standard_normal((m, n)).astype(np.float32)
    with rsvd_lib.Plan(m, n, l - 1, 1, 0, 1) as pl:
        for trans in (0, 1):
            kx = m if trans else n
            x = philox.gaussian(5, 0, kx, l).astype(np.float32)
            Y = torch.zeros((n if trans else m), l, device="cuda")
            rsvd_lib.rsvd_sketch(pl.handle, _dev(a), trans, _dev(x), Y)
            torch.cuda.synchronize()
            a64 = a.astype(np.float64)
            ref = (a64.T if trans else a64) @ x.astype(np.float64)
            bound = 1e-5 * (np.abs(a64.T if trans else a64) @ np.abs(x.astype(np.float64)))
            assert np.all(np.abs(_np(Y) - ref) <= bound)


# --------------------------------------------------------------------------
# step a3: orthonormalisation
# --------------------------------------------------------------------------


def _orth(pkg, y, l, rows, rounds=3):
    with pkg.Plan(rows, rows, l, 0, 0, 0, 0, rounds) as pl:
        Y = _dev(y)
        R = torch.zeros(l, l, device="cuda")
        pkg.rsvd_orthonormalize(pl.handle, rows, Y, R)
        st = pkg.rsvd_sync(pl.handle)
        return _np(Y), _np(R), st


# l_p = 176, 208, 224, 240 and 256 take the row-packed factorisation with a block count
# that is not a multiple of its 4-block load groups (11, 13, 14, 15) or is (16)
@pytest.mark.parametrize("rows,l,cond", [(700, 24, 1e2), (1500, 64, 1e4), (300, 110, 1e3), (5000, 16, 1e5),
                                         (2000, 176, 1e3), (2500, 200, 1e2), (2500, 220, 1e3),
                                         (3000, 236, 1e3), (3000, 250, 1e4), (1024, 256, 1e2)])
def test_orthonormalize_matches_householder(rsvd_lib, rows, l, cond):
    rng = np.random.default_rng(rows)
    y = (synth.haar(rng, rows, l) * np.logspace(0, -np.log10(cond), l)) @ synth.haar(rng, l, l).T
    y = y.astype(np.float32)
    q, r, st = _orth(rsvd_lib, y, l, rows)
    assert st == rsvd_lib.RSVD_OK
    assert metrics.orthonormality(q) <= 1e-5
    qr, rr = rsvd64.qr_pos(y.astype(np.float64))
    # unique QR with diag(R) > 0: elementwise agreement up to cond * u
    assert np.max(np.abs(q - qr)) <= 50 * cond * 6e-8 + 1e-5
    assert np.max(np.abs(r - rr)) <= 1e-5 * np.abs(rr).max() * max(1.0, cond * 1e-3)
    assert np.max(np.abs(q @ r - y)) <= 1e-5 * np.abs(y).max()


@pytest.mark.parametrize("rows,l,r", [(800, 16, 5), (1500, 240, 100)])
def test_orthonormalize_rank_deficient(rsvd_lib, rows, l, r):
    rng = np.random.default_rng(1)
    y = (synth.haar(rng, rows, r) @ rng.standard_normal((r, l))).astype(np.float32)
    q, _, st = _orth(rsvd_lib, y, l, rows)
    assert st == rsvd_lib.RSVD_OK and np.all(np.isfinite(q))
    # the basis still spans range(Y)
    proj = q @ np.linalg.lstsq(q, y.astype(np.float64), rcond=None)[0]
    assert np.max(np.abs(proj - y)) <= 1e-4 * np.abs(y).max()


# --------------------------------------------------------------------------
# step a6: small SVD
# --------------------------------------------------------------------------


_SMALL_CASES = ([(l, 1) for l in (1, 2, 17, 32, 110, 160)] +
                [(l, 2) for l in (1, 2, 17, 63, 110, 129, 160, 192, 255, 256)])


@pytest.mark.parametrize("l,variant", _SMALL_CASES)
def test_small_svd_matches_lapack(rsvd_lib, l, variant):
    """variant 1: one-CTA Jacobi (l <= 160); 2: the 4-CTA cluster Jacobi (l <= 256)."""
    rng = np.random.default_rng(l)
    x = (synth.haar(rng, l, l) * np.logspace(0, -3, l)) @ synth.haar(rng, l, l).T
    x = np.triu(x) if l > 2 else x
    x = x.astype(np.float32)
    with rsvd_lib.Plan(max(l, 2) + 4, max(l, 2) + 4, l, 0, 0, 0, small_svd=variant) as pl:
        Ut = torch.zeros(l, l, device="cuda")
        W = torch.zeros(l, l, device="cuda")
        S = torch.zeros(l, device="cuda")
        rsvd_lib.rsvd_small_svd(pl.handle, _dev(x), Ut, S, W)
        torch.cuda.synchronize()
        bits, sweeps = rsvd_lib.rsvd_diagnostics(pl.handle)
    assert sweeps < 40 and not bits & 16, (bits, sweeps)      # converged before the sweep limit
    ut, s, w = _np(Ut), _np(S), _np(W)
    x64 = x.astype(np.float64)
    uu, ss, vt = np.linalg.svd(x64)
    assert np.all(np.diff(s) <= 0)
    assert np.max(np.abs(s - ss)) <= 1e-5 * ss[0]
    assert np.max(np.abs((ut * s) @ w.T - x64)) <= 1e-5 * ss[0]
    assert metrics.orthonormality(ut) <= 1e-5 and metrics.orthonormality(w) <= 1e-5
    if l <= 160 and variant == 1:
        # the oracle's own Jacobi agrees with LAPACK too (independent route)
        _, sj, _ = ojacobi.jacobi_svd(x64)
        assert np.max(np.abs(sj - ss)) <= 1e-12 * ss[0]


# --------------------------------------------------------------------------
# end to end (a1 .. a7)
# --------------------------------------------------------------------------


def test_rsvd_c1_full_size(rsvd_lib):
    w = synth.C1
    a, *_ = synth.lowrank(w.m, w.n, w.sigma(), w.matrix_seed)
    a32 = a.astype(np.float32)
    u, s, v = _gpu_svd(rsvd_lib, a32, w.k, w.p, w.q, w.omega_seed)
    om = philox.gaussian(w.omega_seed, 0, w.n, w.l)
    _check_svd(a32.astype(np.float64), u, s, v, w.k, w.p, w.q, om)
    assert metrics.orthonormality(u) <= 1e-5 and metrics.orthonormality(v) <= 1e-5


@pytest.mark.parametrize("m,n,k,p,q,rounds", [(517, 389, 12, 7, 1, 3), (389, 517, 12, 7, 0, 3),
                                              (130, 129, 1, 0, 1, 3), (64, 48, 40, 8, 2, 3),
                                              (3000, 40, 10, 5, 1, 2), (257, 1031, 30, 2, 2, 2),
                                              (1100, 900, 236, 20, 1, 3)])
def test_rsvd_shapes_and_ragged_edges(rsvd_lib, m, n, k, p, q, rounds):
    a, *_ = synth.lowrank(m, n, synth.spectrum_exp(min(m, n), 5.0), m * 7 + n)
    a32 = a.astype(np.float32)
    u, s, v = _gpu_svd(rsvd_lib, a32, k, p, q, 77, rounds=rounds)
    om = philox.gaussian(77, 0, n, k + p)
    _check_svd(a32.astype(np.float64), u, s, v, k, p, q, om)


def test_range_finder_matches_oracle(rsvd_lib):
    w = synth.C1
    a, *_ = synth.lowrank(w.m, w.n, w.sigma(), w.matrix_seed)
    a32 = a.astype(np.float32)
    with rsvd_lib.Plan(w.m, w.n, w.k, w.p, w.q, w.omega_seed) as pl:
        Q = pl.range_finder(_dev(a32))
    q = _np(Q)
    om = philox.gaussian(w.omega_seed, 0, w.n, w.l)
    qr = rsvd64.range_finder(a32.astype(np.float64), om, w.q)
    assert metrics.orthonormality(q) <= 1e-5
    # same subspace, and the same columns (unique QR normalisation) up to rounding
    assert np.linalg.norm(q @ (q.T @ qr) - qr, 2) <= 1e-3
    e_gpu = metrics.projection_error(a32.astype(np.float64), q)
    e_ref = metrics.projection_error(a32.astype(np.float64), qr)
    assert abs(e_gpu - e_ref) <= 1e-5 * w.sigma()[0]


def test_exact_rank_recovery(rsvd_lib):
    m, n, r = 900, 600, 10
    sig = np.linspace(2.0, 0.2, r)
    a, *_ = synth.lowrank(m, n, sig, 3)
    a32 = a.astype(np.float32)
    u, s, v = _gpu_svd(rsvd_lib, a32, r, 6, 1, 11)
    assert np.max(np.abs(s - sig)) <= 1e-5 * sig[0]
    assert metrics.fro_error(a32.astype(np.float64), u, s, v) <= 1e-5 * np.linalg.norm(a)


def test_zero_matrix(rsvd_lib):
    a32 = np.zeros((200, 150), np.float32)
    u, s, v = _gpu_svd(rsvd_lib, a32, 5, 3, 1, 1)
    assert np.all(np.abs(s) <= 1e-30) and np.all(np.isfinite(u)) and np.all(np.isfinite(v))


def test_nonfinite_input_is_reported(rsvd_lib):
    a = np.random.default_rng(0).standard_normal((300, 200)).astype(np.float32)
    a[17, 33] = np.nan
    with rsvd_lib.Plan(300, 200, 8, 4, 1, 0) as pl:
        U = torch.empty(300, 8, device="cuda")
        S = torch.empty(8, device="cuda")
        V = torch.empty(200, 8, device="cuda")
        rsvd_lib.rsvd_svd(pl.handle, _dev(a), U, S, V)
        assert rsvd_lib.rsvd_sync(pl.handle) == rsvd_lib.RSVD_ERR_NONFINITE
        assert rsvd_lib.rsvd_sync(pl.handle) == rsvd_lib.RSVD_OK       # cleared


def test_omega_hooks(rsvd_lib):
    m, n, k, p, q = 600, 400, 15, 9, 1
    a, *_ = synth.lowrank(m, n, synth.spectrum_power(n, 1.0), 8)
    a32 = a.astype(np.float32)
    with rsvd_lib.Plan(m, n, k, p, q, 31) as pl:
        O = torch.zeros(n, k + p, device="cuda")
        rsvd_lib.rsvd_get_omega(pl.handle, O)
        torch.cuda.synchronize()
    ref = philox.gaussian(31, 0, n, k + p)
    assert np.all(np.abs(_np(O) - ref) <= 4e-6 * np.maximum(1.0, np.abs(ref)))
    om_user = synth.gaussian_matrix(n, k + p, 99)
    u, s, v = _gpu_svd(rsvd_lib, a32, k, p, q, 31, omega=om_user.astype(np.float32))
    _check_svd(a32.astype(np.float64), u, s, v, k, p, q, om_user.astype(np.float32).astype(np.float64))


def test_host_buffer_entry_point(rsvd_lib):
    m, n, k, p, q = 700, 500, 10, 5, 1
    a, *_ = synth.lowrank(m, n, synth.spectrum_exp(n, 7.0), 4)
    a32 = torch.tensor(a.astype(np.float32)).pin_memory()
    with rsvd_lib.Plan(m, n, k, p, q, 5) as pl:
        Uh = torch.empty(m, k).pin_memory()
        Sh = torch.empty(k).pin_memory()
        Vh = torch.empty(n, k).pin_memory()
        rsvd_lib.rsvd_svd_host(pl.handle, a32, Uh, Sh, Vh)
        U, S, V = pl.svd(a32.cuda())
    assert np.array_equal(Sh.numpy(), S.cpu().numpy())
    assert np.array_equal(Uh.numpy(), U.cpu().numpy())


def test_c2_full_size_fp32(rsvd_lib):
    """Config C2 at full size (16384^2, sigma_j = j^-1.5, k=100, p=10, q=1), plain FP32 path."""
    w = synth.C2
    A = synth.device_lowrank(w.m, w.n, w.sigma(), w.matrix_seed)
    with rsvd_lib.Plan(w.m, w.n, w.k, w.p, w.q, w.omega_seed) as pl:
        U, S, V = pl.svd(A)
    a64 = A.cpu().numpy().astype(np.float64)
    del A
    om = philox.gaussian(w.omega_seed, 0, w.n, w.l)
    _check_svd(a64, _np(U), _np(S), _np(V), w.k, w.p, w.q, om)


@pytest.mark.parametrize("m", [701, 61])
def test_host_f32_entry_point_splits_like_the_device(rsvd_lib, m):
    """rsvd_svd_host with host_f32 = 1 and A stored as hi + lo: the float32 A is copied in
    four pieces of rows (uneven here: 701 = 3 x 176 + 173, 61 = 3 x 16 + 13)
    and each piece split into hi + lo on its own stream; the result must equal, bit for
    bit, rsvd_svd on the device split of the same A."""
    n, k, p, q = 512, 10, 6, 1
    a, *_ = synth.lowrank(m, n, synth.spectrum_exp(min(m, n), 7.0), 14)
    a32 = torch.tensor(a.astype(np.float32)).pin_memory()
    with rsvd_lib.Plan(m, n, k, p, q, 5, rsvd_lib.RSVD_BF16_TC, dtype=rsvd_lib.RSVD_BF16X2,
                       residual_passes=1, host_f32=1) as pl:
        Uh = torch.empty(m, k).pin_memory()
        Sh = torch.empty(k).pin_memory()
        Vh = torch.empty(n, k).pin_memory()
        rsvd_lib.rsvd_svd_host(pl.handle, a32, Uh, Sh, Vh)
        U, S, V = pl.svd(rsvd_lib.split_bf16(a32.cuda()))
        assert rsvd_lib.rsvd_sync(pl.handle) == rsvd_lib.RSVD_OK
    assert np.array_equal(Sh.numpy(), S.cpu().numpy())
    assert np.array_equal(Uh.numpy(), U.cpu().numpy())
    assert np.array_equal(Vh.numpy(), V.cpu().numpy())
