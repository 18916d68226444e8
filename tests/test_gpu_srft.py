"""GPU parity of the SRFT test matrix (Section 4.6, Algorithm 4.5) against the oracle.

Omega from the library (rsvd_get_omega) is compared element by element with the
oracle's explicit real SRFT built from the same Philox draws: signs and sampled
frequencies are integer decisions, so a wrong one shows up as an O(1) error; the
float32 cos/sin of exactly reduced angles agree to a few ulp (<= 2e-6 / sqrt(l_c)).
The full randomized SVD with the SRFT is then held to the same tolerances as the
Gaussian path, against the oracle run with that Omega.
"""
import os
import sys

import numpy as np
import pytest
import torch

from oracle import metrics, srft

sys.path.insert(0, os.path.dirname(__file__))
from test_gpu_parity import _check_svd, _dev, _np  # noqa: E402

pytestmark = pytest.mark.gpu


def _srft_plan(pkg, m, n, k, p, q, seed, precision=0):
    return pkg.Plan(m, n, k, p, q, seed, precision, test_matrix=pkg.RSVD_SRFT)


@pytest.mark.parametrize("m,n,l,seed", [(16, 64, 8, 5), (40, 1000, 30, 2004), (200, 4096, 128, 77),
                                        (256, 32768, 256, 2004), (300, 514, 256, 1)])
def test_srft_omega_matches_oracle(rsvd_lib, m, n, l, seed):
    with _srft_plan(rsvd_lib, m, n, l - 2, 2, 1, seed) as pl:
        om = torch.zeros(n, l, device="cuda")
        rsvd_lib.rsvd_get_omega(pl.handle, om)
        torch.cuda.synchronize()
    got = _np(om)
    signs, freqs = srft.draw(seed, n, l // 2)
    ref = srft.omega_real(signs, freqs)
    assert np.max(np.abs(got - ref)) <= 2e-6 / np.sqrt(l // 2) + 1e-7
    # structure: the columns are orthogonal with norm^2 n / (2 l_c) each (Omega^H Omega = (n/l_c) I
    # for the complex matrix; real and imaginary parts split it evenly for 0 < b < n/2)
    g = got.T @ got
    assert np.allclose(g, np.eye(l) * n / l, atol=2e-4 * n / l)


@pytest.mark.parametrize("m,n,k,p,q", [(700, 512, 20, 12, 1), (1000, 2048, 100, 28, 1), (517, 390, 8, 4, 2)])
def test_srft_rsvd_fp32_matches_oracle(rsvd_lib, m, n, k, p, q):
    import synth

    a, *_ = synth.lowrank(m, n, synth.spectrum_power(min(m, n), 0.5), m + 3 * n)
    a32 = a.astype(np.float32)
    seed = 31
    with _srft_plan(rsvd_lib, m, n, k, p, q, seed) as pl:
        om = torch.zeros(n, k + p, device="cuda")
        rsvd_lib.rsvd_get_omega(pl.handle, om)
        U, S, V = pl.svd(_dev(a32))
        torch.cuda.synchronize()
    u, s, v = _np(U), _np(S), _np(V)
    signs, freqs = srft.draw(seed, n, (k + p) // 2)
    omega = srft.omega_real(signs, freqs)
    assert np.max(np.abs(_np(om) - omega)) <= 2e-6
    _check_svd(a32.astype(np.float64), u, s, v, k, p, q, omega)
    assert metrics.orthonormality(u) <= 1e-5 and metrics.orthonormality(v) <= 1e-5


def test_srft_sketch_is_the_fft_sketch(rsvd_lib):
    """Y = A Omega through the library's pass equals the row-FFT form of Algorithm 4.5."""
    rng = np.random.default_rng(3)
    m, n, l = 300, 1024, 64
    a32 = rng.standard_normal((m, n)).astype(np.float32)
    with _srft_plan(rsvd_lib, m, n, l - 4, 4, 0, 11) as pl:
        om = torch.zeros(n, l, device="cuda")
        rsvd_lib.rsvd_get_omega(pl.handle, om)
        Y = torch.zeros(m, l, device="cuda")
        rsvd_lib.rsvd_sketch(pl.handle, _dev(a32), 0, om, Y)
        torch.cuda.synchronize()
    signs, freqs = srft.draw(11, n, l // 2)
    ref = srft.sketch_fft(a32.astype(np.float64), signs, freqs)
    scale = np.abs(a32).astype(np.float64) @ np.abs(srft.omega_real(signs, freqs))
    assert np.all(np.abs(_np(Y) - ref) <= 1e-5 * scale + 1e-6)


@pytest.mark.parametrize("m,n,l,kind", [(300, 2048, 64, "f32"), (257, 4096, 128, "f32"), (130, 8192, 32, "bf16"),
                                        (96, 16384, 40, "f32"), (300, 32768, 256, "f32"), (260, 32768, 256, "hilo")])
def test_srft_row_transform_matches_oracle(rsvd_lib, m, n, l, kind):
    """The row-transform sketch (signs, a length-n FFT per row in shared memory, the sampled
    frequencies) against the oracle's full-FFT form of Algorithm 4.5 on the stored A.  An
    FFT's rounding error per output is about log2(n) u32 ||row||_2 (times the output scale
    l_c^-1/2): the bound allows 8 log2(n) u32 ||row||_2 / sqrt(l_c)."""
    pkg = rsvd_lib
    rng = np.random.default_rng(n + l)
    a32 = (rng.standard_normal((m, n)) * np.exp(rng.standard_normal((m, 1)))).astype(np.float32)
    seed = 2004
    kw = {}
    if kind == "bf16":
        kw = dict(precision=pkg.RSVD_BF16_TC, dtype=pkg.RSVD_BF16)
    elif kind == "hilo":
        kw = dict(precision=pkg.RSVD_BF16_TC, dtype=pkg.RSVD_BF16X2, residual_passes=1)
    with pkg.Plan(m, n, l - 4, 4, 0, seed, test_matrix=pkg.RSVD_SRFT, **kw) as pl:
        A = pl.stored(_dev(a32))
        Y = torch.full((m, l), float("nan"), device="cuda")
        pkg.rsvd_sketch_srft(pl.handle, A, Y)
        assert pkg.rsvd_sync(pl.handle) == pkg.RSVD_OK
        a_st = _np(A)
    if kind == "hilo":
        a_st = a_st[:m] + a_st[m:]
    signs, freqs = srft.draw(seed, n, l // 2)
    ref = srft.sketch_fft(a_st, signs, freqs)
    tol = 8 * np.log2(n) * 2.0 ** -24 * np.linalg.norm(a_st, axis=1, keepdims=True) / np.sqrt(l // 2)
    err = np.abs(_np(Y) - ref)
    print(f"srft row transform n={n} l={l} {kind}: max err / tol {np.max(err / tol):.3f}")
    assert np.all(err <= tol)


def test_srft_row_transform_is_the_plans_first_pass(rsvd_lib):
    """rsvd_range_finder on an SRFT plan with n = 4096 and srft_fft = 1 takes the row
    transform; setting the same Omega explicitly takes the dense pass: the two bases agree
    to float32 rounding."""
    import synth

    pkg = rsvd_lib
    m, n, k, p, q = 900, 4096, 40, 24, 1
    a, *_ = synth.lowrank(m, n, synth.spectrum_power(min(m, n), 0.5), 5)
    A = _dev(a.astype(np.float32))
    with pkg.Plan(m, n, k, p, q, 7, test_matrix=pkg.RSVD_SRFT, srft_fft=1) as pl:
        Q1 = pl.range_finder(A)
        om = torch.zeros(n, k + p, device="cuda")
        pkg.rsvd_get_omega(pl.handle, om)
        pkg.rsvd_set_omega(pl.handle, om)
        Q2 = pl.range_finder(A)
    assert torch.max(torch.abs(Q1 - Q2)).item() <= 1e-4


# ---- the modified SRFT (Section 4.6, eq. random_Givens)
#
# The two Givens chains carry one running value down n - 1 rotations each, so float32
# rounding accumulates like a random walk: |Omega_gpu - Omega_ref| <= 2 u sqrt(2 n) of
# the largest entry (u = 2^-24; the angles are float32 sincospi of exactly representable
# arguments).  The permutations and signs are integer decisions: a wrong one is an O(1)
# error.

@pytest.mark.parametrize("n,l,seed", [(64, 8, 5), (1024, 80, 3), (4096, 160, 9), (2050, 256, 1)])
def test_gsrft_omega_matches_oracle(rsvd_lib, n, l, seed):
    pkg = rsvd_lib
    with pkg.Plan(l + 8, n, l - 2, 2, 0, seed, test_matrix=pkg.RSVD_GSRFT) as pl:
        om = torch.zeros(n, l, device="cuda")
        pkg.rsvd_get_omega(pl.handle, om)
        assert pkg.rsvd_sync(pl.handle) == pkg.RSVD_OK
    got = _np(om)
    ref = srft.gsrft_omega_real(seed, n, l // 2)
    tol = 2 * 2.0 ** -24 * np.sqrt(2 * n) * np.abs(ref).max()
    err = np.max(np.abs(got - ref))
    print(f"GSRFT n={n} l={l}: max error {err:.2e} (tolerance {tol:.2e})")
    assert err <= tol
    assert np.allclose(got.T @ got, np.eye(l) * n / l, atol=2e-4 * n / l)


@pytest.mark.parametrize("m,n,k,p,q,prec", [(700, 512, 20, 12, 1, 0), (1024, 1024, 80, 0, 0, 0),
                                            (1500, 2048, 100, 28, 1, 1)])
def test_gsrft_rsvd_matches_oracle(rsvd_lib, m, n, k, p, q, prec):
    """The whole randomized SVD with the modified SRFT (plain path: the float32 targets
    against the oracle run with the oracle's Omega; tensor-core path: the reconstruction
    error within 1e-3 of the oracle's, as the bfloat16 operands move it by design)."""
    import synth

    pkg = rsvd_lib
    a, *_ = synth.lowrank(m, n, synth.spectrum_power(min(m, n), 0.5), m + 5 * n)
    a32 = a.astype(np.float32)
    seed = 41
    l = k + p
    omega = srft.gsrft_omega_real(seed, n, l // 2)
    tc = prec == pkg.RSVD_BF16_TC
    with pkg.Plan(m, n, k, p, q, seed, prec, test_matrix=pkg.RSVD_GSRFT) as pl:
        A = _dev(a32)
        if tc:
            A = A.to(torch.bfloat16)
        U, S, V = pl.svd(A)
        torch.cuda.synchronize()
    u, s, v = _np(U), _np(S), _np(V)
    a64 = (A.float().cpu().numpy() if tc else a32).astype(np.float64)
    if not tc:
        _check_svd(a64, u, s, v, k, p, q, omega)
    else:
        from oracle import rsvd64

        ur, sr, vr, _ = rsvd64.rsvd(a64, k, p, q, omega)
        e_ref = metrics.fro_error_onepass(a64, ur, sr, vr)
        e_gpu = metrics.fro_error_onepass(a64, u, s, v)
        assert abs(e_gpu - e_ref) <= 1e-3 * e_ref
    assert metrics.orthonormality(u) <= 2e-5 and metrics.orthonormality(v) <= 2e-5
