"""Pins of the float64 oracle against facts the paper and mathematics fix (CPU only).

Each test names the passage it checks.  Together they are chosen so that a
plausible slip in the oracle (a dropped term, a transposed operand, a wrong
sign or index) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import synth
from oracle import bounds, grad, jacobi, metrics, philox, rsvd64, single_pass, srft

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# test matrix generator (Algorithm 4.1 step 1)
# --------------------------------------------------------------------------


def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(w, 16) for w in line.split()])
    for r in rows:
        out = philox.philox4x32_10(np.array([r[:4]], np.uint32), np.array(r[4:6], np.uint32))[0]
        assert [int(x) for x in out] == r[6:]


def test_uniforms_open_interval_and_exact():
    u = philox.bits_to_uniform(np.array([0, 0xFFFFFFFF, 511, 512], np.uint32))
    assert u[0] == 2.0 ** -24 and u[1] == 1.0 - 2.0 ** -24
    assert u[2] == u[0] and u[3] == 3 * 2.0 ** -24
    assert np.all(u.astype(np.float32).astype(np.float64) == u)


def test_gaussian_layout_and_moments():
    z = philox.gaussian(7, philox.STREAM_OMEGA, 5000, 40)
    assert z.shape == (5000, 40)
    # column 4g+t of row i comes from counter (g, i, stream, 0), word t
    w = philox.raw_words(7, 0, 5000, 10)
    u = philox.bits_to_uniform(w[3, 2])
    zz = math.sqrt(-2 * math.log(u[2])) * math.sin(2 * math.pi * u[3])
    assert z[3, 11] == pytest.approx(zz, abs=1e-14)
    x = z.ravel()
    assert abs(x.mean()) < 4 / math.sqrt(x.size)
    assert abs(x.var() - 1.0) < 4 * math.sqrt(2.0 / x.size)
    from scipy import stats

    assert stats.kstest(x, "norm").pvalue > 1e-3
    # distinct streams and seeds give independent draws
    z2 = philox.gaussian(7, philox.STREAM_PSI, 5000, 40)
    assert abs(np.corrcoef(z.ravel(), z2.ravel())[0, 1]) < 0.02


def test_pinv_gaussian_moments():
    """Proposition 10.2: E||G^+||_F^2 = k/(p-1) and E||G^+|| <= e sqrt(k+p)/p."""
    k, p, trials = 10, 10, 10000
    z = philox.gaussian(11, philox.STREAM_OMEGA, trials * k, k + p).reshape(trials, k, k + p)
    ggt = z @ np.transpose(z, (0, 2, 1))
    inv = np.linalg.inv(ggt)
    fro2 = np.trace(inv, axis1=1, axis2=2)                 # ||G^+||_F^2 = tr((G G^T)^-1)
    se = fro2.std() / math.sqrt(trials)
    assert abs(fro2.mean() - bounds.pinv_gauss_frobenius_mean(k, p)) < 4 * se
    spec = np.sqrt(np.linalg.eigvalsh(inv)[:, -1])
    assert spec.mean() <= bounds.pinv_gauss_spectral_mean(k, p)


# --------------------------------------------------------------------------
# QR convention and Stage A (Algorithms 4.1, 4.3, 4.4)
# --------------------------------------------------------------------------


def test_qr_pos():
    y = synth.gaussian_matrix(300, 25, 3) @ np.diag(np.logspace(0, -4, 25))
    q, r = rsvd64.qr_pos(y)
    assert metrics.orthonormality(q) < 1e-13
    assert np.all(np.diag(r) > 0) and np.allclose(np.tril(r, -1), 0)
    assert np.max(np.abs(q @ r - y)) < 1e-13 * np.max(np.abs(y))


@pytest.mark.parametrize("q", [0, 1, 2])
def test_exact_rank_recovery(q):
    """Exact rank r <= k: the sample spans range(A) and the error vanishes (Section 1.3, Theorem 9.1 proof)."""
    m, n, r, k, p = 300, 200, 10, 10, 5
    sig = np.linspace(3.0, 0.5, r)
    a, u, s, v = synth.lowrank(m, n, sig, 21)
    om = philox.gaussian(5, 0, n, k + p)
    qm = rsvd64.range_finder(a, om, q)
    assert metrics.projection_error(a, qm) <= 1e-13 * np.linalg.norm(a, 2)
    uu, ss, vv, _ = rsvd64.rsvd(a, k, p, q, om)
    assert np.max(np.abs(ss - sig) / sig[0]) < 1e-13
    assert metrics.fro_error(a, uu, ss, vv) < 1e-12 * np.linalg.norm(a)


@pytest.mark.parametrize("q", [0, 2])
def test_orthonormal_bases(q):
    w = synth.C1
    a, *_ = synth.lowrank(w.m // 4, w.n // 4, w.sigma()[: w.n // 4], 4)
    om = philox.gaussian(9, 0, a.shape[1], w.l)
    qm, steps = rsvd64.range_finder(a, om, q, keep_steps=True)
    assert len(steps) == 2 * q + 1
    for s in steps:
        assert metrics.orthonormality(s) < 1e-13


def _case(seed, m=240, n=160, rate=6.0):
    sig = synth.spectrum_exp(min(m, n), rate)
    return synth.lowrank(m, n, sig, seed)


@pytest.mark.parametrize("seed", range(6))
def test_deterministic_bound_theorem_9_1(seed):
    """Theorem 9.1, spectral and Frobenius norms, every instance (no probability involved)."""
    a, u, s, v = _case(seed)
    for k, p in ((8, 4), (15, 0), (20, 10)):
        om = philox.gaussian(100 + seed, 0, a.shape[1], k + p)
        qm = rsvd64.range_finder(a, om, 0)
        for norm in ("2", "fro"):
            err = metrics.projection_error(a, qm, norm)
            assert err <= bounds.deterministic(s, v, om, k, norm) * (1 + 1e-9) + 1e-14


@pytest.mark.parametrize("q", [1, 2])
def test_power_scheme_theorems_9_1_and_9_2(q):
    """Theorem 9.2 with Z = (AA^T)^q A Omega, and Theorem 9.1 applied to (AA^T)^q A."""
    a, u, s, v = _case(31, rate=10.0)
    k, p = 10, 5
    om = philox.gaussian(77, 0, a.shape[1], k + p)
    qm = rsvd64.range_finder(a, om, q)
    b = np.linalg.matrix_power(a @ a.T, q) @ a
    lhs = metrics.projection_error(a, qm)
    mid = metrics.projection_error(b, qm) ** (1.0 / (2 * q + 1))
    assert lhs <= mid * (1 + 1e-9)
    rhs = bounds.deterministic(s ** (2 * q + 1), v, om, k) ** (1.0 / (2 * q + 1))
    assert mid <= rhs * (1 + 1e-6)


def test_power_spectrum_and_algorithm_4_3_equivalence():
    """sigma_j((AA^T)^q A) = sigma_j^(2q+1) (Section 4.5); Alg 4.3 and 4.4 span the same range in exact arithmetic."""
    a, u, s, v = _case(5, m=120, n=80, rate=40.0)
    for q in (1, 2):
        b = np.linalg.matrix_power(a @ a.T, q) @ a
        sb = np.linalg.svd(b, compute_uv=False)[: len(s)]
        assert np.allclose(sb, s ** (2 * q + 1), rtol=1e-10, atol=1e-14 * sb[0])
        om = philox.gaussian(3, 0, 80, 12)
        q3 = rsvd64.power_iteration(a, om, q)
        q4 = rsvd64.range_finder(a, om, q)
        assert np.max(np.abs(q3 @ q3.T - q4 @ q4.T)) < 1e-8


def test_truncation_theorem_9_3_and_no_degradation():
    """Algorithm 5.1 keeps the range-finder error (Section 5.1); Theorem 9.3 bounds the truncated SVD."""
    a, u, s, v = _case(8, rate=5.0)
    for k, p, q in ((10, 10, 0), (12, 6, 1)):
        om = philox.gaussian(41, 0, a.shape[1], k + p)
        qm = rsvd64.range_finder(a, om, q)
        uf, sf, vf = rsvd64.direct_svd(a, qm)
        err_q = metrics.projection_error(a, qm)
        err_full = np.linalg.norm(a - (uf * sf) @ vf.T, 2)
        assert abs(err_full - err_q) <= 1e-12 * s[0]
        assert metrics.orthonormality(uf) < 1e-13 and metrics.orthonormality(vf) < 1e-13
        ut, st, vt = rsvd64.truncate(uf, sf, vf, k)
        err_t = np.linalg.norm(a - (ut * st) @ vt.T, 2)
        assert err_t <= s[k] + err_q + 1e-13
        # the truncation is a best rank-k approximation of P_Q A
        pa = qm @ (qm.T @ a)
        sv = np.linalg.svd(pa, compute_uv=False)
        assert np.allclose(st, sv[:k], rtol=1e-11)


def test_average_error_bounds_over_seeds():
    """Theorems 1.1, 10.5, 10.6, Corollary 10.10 (means) and the 11 sqrt bound (every trial)."""
    m, n, k, p = 400, 200, 20, 10
    sig = synth.spectrum_exp(n, 8.0)
    a, u, s, v = synth.lowrank(m, n, sig, 12)
    trials = 120
    e2 = {0: [], 2: []}
    ef = []
    for t in range(trials):
        om = philox.gaussian(5000 + t, 0, n, k + p)
        for q in (0, 2):
            qm = rsvd64.range_finder(a, om, q)
            e2[q].append(metrics.projection_error(a, qm))
            if q == 0:
                ef.append(metrics.projection_error(a, qm, "fro"))
    e0 = np.array(e2[0])
    assert e0.mean() <= bounds.avg_spectral(k, p, s)
    assert e0.mean() <= bounds.intro_expectation(k, p, m, n, s[k])
    assert np.mean(ef) <= bounds.avg_frobenius(k, p, s)
    assert np.all(e0 <= bounds.intro_probability(k, p, m, n, s[k]))
    assert np.mean(e2[2]) <= bounds.avg_spectral_power(k, p, 2, s)
    assert np.all(e0 >= s[k + p] * (1 - 1e-12))       # a rank-(k+p) basis never beats sigma_{k+p+1} (Mirsky)
    assert np.mean(e2[2]) < e0.mean()                    # the power scheme helps


def test_rank_2k_power_scheme_bound_theorem_1_2():
    m, n, k, q = 300, 200, 10, 1
    sig = synth.spectrum_power(n, 0.8)
    a, u, s, v = synth.lowrank(m, n, sig, 13)
    errs = []
    for t in range(40):
        om = philox.gaussian(900 + t, 0, n, 2 * k)
        uu, ss, vv, _ = rsvd64.rsvd(a, 2 * k, 0, q, om)
        errs.append(np.linalg.norm(a - (uu * ss) @ vv.T, 2))
    assert np.mean(errs) <= bounds.intro_rsvd_expectation(k, q, m, n, s[k])


# --------------------------------------------------------------------------
# Stage B small SVD (Algorithm 5.1 step 2, Section 3.3.3)
# --------------------------------------------------------------------------


@pytest.mark.parametrize("seed", [0, 1])
def test_jacobi_svd_against_lapack(seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((40, 40)) @ np.diag(np.logspace(0, -6, 40)) @ synth.haar(rng, 40, 40).T
    u, s, v = jacobi.jacobi_svd(x)
    s_ref = np.linalg.svd(x, compute_uv=False)
    assert np.max(np.abs(s - s_ref)) < 1e-13 * s_ref[0]
    assert metrics.orthonormality(u) < 1e-12 and metrics.orthonormality(v) < 1e-12
    assert np.max(np.abs((u * s) @ v.T - x)) < 1e-13 * s_ref[0]


def test_stage_b_via_qr_of_bt_matches_direct():
    a, *_ = _case(17, rate=7.0)
    k, p, q = 12, 8, 1
    om = philox.gaussian(2, 0, a.shape[1], k + p)
    u1, s1, v1, _ = rsvd64.rsvd(a, k, p, q, om)
    for small in (None, jacobi.jacobi_svd):
        u2, s2, v2, _ = rsvd64.rsvd_via_qr_of_bt(a, k, p, q, om, small_svd=small)
        assert np.max(np.abs(s1 - s2)) < 1e-13 * s1[0]
        assert np.max(np.abs(metrics.align_columns(u1, u2) - u1)) < 1e-9
        assert np.max(np.abs(metrics.align_columns(v1, v2) - v1)) < 1e-9


# --------------------------------------------------------------------------
# SRFT (Section 4.6, Algorithm 4.5, Section 11.1 norm identity)
# --------------------------------------------------------------------------


def test_srft_structure():
    n, lc = 64, 12
    d, f = srft.draw(3, n, lc)
    assert set(np.unique(d)) <= {-1.0, 1.0}
    assert len(set(f.tolist())) == lc and f.min() >= 1 and f.max() <= n // 2 - 1
    om = srft.omega_complex(d, f)
    assert np.max(np.abs(om.conj().T @ om - (n / lc) * np.eye(lc))) < 1e-12
    assert np.linalg.norm(om, 2) == pytest.approx(math.sqrt(n / lc), rel=1e-12)
    omr = srft.omega_real(d, f)
    assert np.max(np.abs(omr.T @ omr - n / (2 * lc) * np.eye(2 * lc))) < 1e-12
    assert np.allclose(omr[:, 0::2], om.real) and np.allclose(omr[:, 1::2], om.imag)


def test_srft_fft_sketch_equals_dense_dft():
    rng = np.random.default_rng(4)
    n, lc = 64, 10
    a = rng.standard_normal((30, n))
    d, f = srft.draw(8, n, lc)
    ref = a @ srft.omega_real(d, f)
    assert np.max(np.abs(srft.sketch_fft(a, d, f) - ref)) < 1e-12
    yc = a @ srft.omega_complex(d, f)
    assert np.max(np.abs(srft.sketch_fft(a, d, f)[:, 0::2] - yc.real)) < 1e-12


def test_srft_draw_is_uniform_subset():
    counts = np.zeros(31)
    for s in range(400):
        _, f = srft.draw(s, 64, 6)
        counts[f - 1] += 1
    expected = 400 * 6 / 31
    assert np.all(np.abs(counts - expected) < 5 * math.sqrt(expected))


# --------------------------------------------------------------------------
# single pass (Section 5.5)
# --------------------------------------------------------------------------


def test_single_pass_solver_matches_bruteforce():
    rng = np.random.default_rng(6)
    l, lt = 5, 4
    x1, c1 = rng.standard_normal((lt, 7)), rng.standard_normal((l, 7))
    x2, c2 = rng.standard_normal((l, 6)), rng.standard_normal((lt, 6))
    b1 = single_pass.min_residual(x1, c1, x2, c2)
    b2 = single_pass.min_residual_bruteforce(x1, c1, x2, c2)
    assert np.max(np.abs(b1 - b2)) < 1e-10
    # normal equations hold
    res = (x2 @ x2.T) @ b1 + b1 @ (x1 @ x1.T) - (c1 @ x1.T + x2 @ c2.T)
    assert np.max(np.abs(res)) < 1e-10


def test_single_pass_exact_rank_and_consistency():
    m, n, r, l = 200, 150, 8, 12
    a, u, s, v = synth.lowrank(m, n, np.linspace(2, 0.3, r), 9)
    om = philox.gaussian(1, philox.STREAM_OMEGA, n, l)
    ps = philox.gaussian(1, philox.STREAM_PSI, m, l)
    uu, ss, vv, (qm, qt, b) = single_pass.rsvd_single_pass(a, r, om, ps)
    assert np.max(np.abs(ss - s)) < 1e-12 * s[0]
    assert metrics.fro_error(a, uu, ss, vv) < 1e-11
    # with exact B = Q^T A Qt both relations hold exactly
    assert np.allclose(b, qm.T @ a @ qt, atol=1e-12)


def test_single_pass_truncated_bases_reduce_to_the_square_form_at_p0():
    """With p = 0 the k leading left singular vectors span range(Y): same B up to the basis."""
    m, n, k = 300, 200, 10
    a, *_ = synth.lowrank(m, n, synth.spectrum_exp(n, 6.0), 13)
    om = philox.gaussian(2, philox.STREAM_OMEGA, n, k)
    ps = philox.gaussian(2, philox.STREAM_PSI, m, k)
    u1, s1, v1, _ = single_pass.rsvd_single_pass(a, k, om, ps, truncate_bases=True)
    u2, s2, v2, _ = single_pass.rsvd_single_pass(a, k, om, ps, truncate_bases=False)
    assert np.max(np.abs(s1 - s2)) < 1e-10 * s2[0]
    assert np.allclose(u1 @ np.diag(s1) @ v1.T, u2 @ np.diag(s2) @ v2.T, atol=1e-10 * s2[0])


def test_single_pass_truncated_bases_on_a_noisy_flat_tail():
    """The remark on single-pass error (Section 5.5): on a noisy, slowly decaying spectrum
    the square system degrades the approximation; the overdetermined k x l system keeps it
    within a small factor of the two-pass error."""
    m, n, k, p = 4096, 512, 32, 8
    sig = np.maximum(np.exp(-np.arange(n) / 10.0), 1e-6)
    a, *_ = synth.lowrank(m, n, sig, 21)
    a = a + 1e-4 * np.random.default_rng(3).standard_normal((m, n))
    om = philox.gaussian(5, philox.STREAM_OMEGA, n, k + p)
    ps = philox.gaussian(5, philox.STREAM_PSI, m, k + p)
    e = {}
    for t in (True, False):
        u, s, v, _ = single_pass.rsvd_single_pass(a, k, om, ps, truncate_bases=t)
        e[t] = metrics.fro_error(a, u, s, v)
    u2, s2, v2, _ = rsvd64.rsvd(a, k, p, 0, om)
    e_two = metrics.fro_error(a, u2, s2, v2)
    assert e[True] < 0.5 * e[False]
    assert e[True] < 10.0 * e_two


# --------------------------------------------------------------------------
# gradient of the reconstruction loss, Omega fixed
# --------------------------------------------------------------------------


def test_gradient_autograd_vs_full_finite_differences():
    m, n, k, p, q = 8, 6, 2, 2, 1
    a, *_ = synth.lowrank(m, n, np.array([3.0, 1.5, 0.6, 0.25, 0.1, 0.04]), 2)
    om = philox.gaussian(4, 0, n, k + p)
    g_ad = grad.grad_autograd(a, k, p, q, om)
    g_fd = grad.grad_fd(a, k, p, q, om, h=1e-3)
    assert np.max(np.abs(g_ad - g_fd)) < 1e-5 * np.max(np.abs(g_ad))


def test_gradient_directional_and_closed_form():
    m, n, k, p, q = 60, 40, 6, 4, 3
    sig = 0.3 ** np.arange(min(m, n))
    sig[:k] = np.linspace(4.0, 1.0, k)
    a, *_ = synth.lowrank(m, n, sig, 3)
    om = philox.gaussian(6, 0, n, k + p)
    g_ad = grad.grad_autograd(a, k, p, q, om)
    rng = np.random.default_rng(0)
    dirs = [e / np.linalg.norm(e) for e in rng.standard_normal((6, m, n))]
    fd = grad.grad_fd(a, k, p, q, om, h=1e-3, directions=dirs)
    ad = np.array([np.sum(g_ad * e) for e in dirs])
    assert np.max(np.abs(fd - ad)) < 1e-5 * np.linalg.norm(g_ad)
    g_cf = grad.grad_exact_svd(a, k)
    # the dominant subspace is captured to ~ (sigma_{k+1}/sigma_k)^(2q+1): close to the exact-SVD gradient
    assert np.linalg.norm(g_ad - g_cf) < 1e-3 * np.linalg.norm(g_cf)


# --------------------------------------------------------------------------
# metrics
# --------------------------------------------------------------------------


def test_error_identities():
    a, *_ = _case(2)
    om = philox.gaussian(3, 0, a.shape[1], 15)
    u, s, v, _ = rsvd64.rsvd(a, 10, 5, 1, om)
    assert metrics.fro_error_onepass(a, u, s, v) == pytest.approx(metrics.fro_error(a, u, s, v), rel=1e-9)
    r = a - (u * s) @ v.T
    assert metrics.spec_norm(r, iters=300) == pytest.approx(metrics.spec_norm(r), rel=1e-6)
    d = np.where(np.arange(u.shape[1]) % 2, -1.0, 1.0)     # flip every other singular pair
    uc, vc = metrics.canonical_signs(u * d, v * d)
    u0, v0 = metrics.canonical_signs(u, v)
    assert np.allclose(uc, u0) and np.allclose(vc, v0)
    assert np.allclose((uc * s) @ vc.T, (u * s) @ v.T)


def test_cotangent_gradient_autograd_vs_finite_differences():
    """General cotangents <gU, U> + <gS, S> + <gV, V> through Algorithm 4.4 + 5.1 (Omega
    fixed): torch autograd of the float64 steps against central differences along random
    directions; the sign of each singular pair is held to the unperturbed branch."""
    rng = np.random.default_rng(21)
    m, n, k, p, q = 14, 11, 3, 2, 1
    a, *_ = synth.lowrank(m, n, np.array([5.0, 3.0, 2.0, 1.2, 0.7, 0.4, 0.2, 0.1, 0.05, 0.02, 0.01]), 4)
    om = rng.standard_normal((n, k + p))
    gu, gs, gv = rng.standard_normal((m, k)), rng.standard_normal(k), rng.standard_normal((n, k))
    g_ad, u, s, v = grad.cotangent_autograd(a, k, p, q, om, gu, gs, gv)
    u0, s0, v0, _ = rsvd64.rsvd(a, k, p, q, om)
    assert np.allclose(s, s0, rtol=1e-13)
    assert np.allclose(np.abs(np.sum(u * u0, axis=0)), 1.0, atol=1e-10)   # same factors up to sign
    dirs = [rng.standard_normal((m, n)) for _ in range(6)]
    fd = grad.cotangent_fd(a, k, p, q, om, gu, gs, gv, dirs, h=1e-5, ref=(u, v))
    ad = np.array([np.sum(g_ad * e) for e in dirs])
    assert np.allclose(ad, fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())
    # gS alone gives d sigma_i = u_i^T dA v_i on the exact-rank part (p large enough):
    # the randomized sigma_i are the Ritz values on the sampled subspace
    g_s, *_ = grad.cotangent_autograd(a, k, p, q, om, 0 * gu, np.eye(k)[0], 0 * gv)
    fd1 = grad.cotangent_fd(a, k, p, q, om, 0 * gu, np.eye(k)[0], 0 * gv, dirs[:2], h=1e-5, ref=(u, v))
    assert np.allclose([np.sum(g_s * e) for e in dirs[:2]], fd1, rtol=1e-5, atol=1e-8)


def test_single_pass_wide_psi_on_the_noisy_tall_workload():
    """Reading of Section 5.5 for the tall-skinny workload: the width l' of Psi is open.  At
    the workload's noise level (noise Frobenius norm equal to the signal's), with l' = l
    the minimum-residual B is worse than the zero matrix (relative error above 1), with
    l' = 3 l the system for B^T is overdetermined enough to bring it below 1, while two
    passes with q = 2 stay the reference (the section's remark: one pass costs accuracy)."""
    m, n, k, p = 16384, 1024, 64, 16
    sig = synth.spectrum_exp_floor(n, 20.0, 1e-6)
    a, *_ = synth.lowrank(m, n, sig, 1003)
    a += synth.noise(m, n, float(np.sqrt(np.sum(sig ** 2) / (m * n))), 77)
    nrm = np.linalg.norm(a)
    om = philox.gaussian(2003, 0, n, k + p)

    def rel(u, s, v):
        return np.linalg.norm(a - (u * s) @ v.T) / nrm

    e_q2 = rel(*rsvd64.rsvd(a, k, p, 2, om)[:3])
    e_l = rel(*single_pass.rsvd_single_pass(a, k, om, philox.gaussian(2003, 1, m, k + p))[:3])
    e_3l = rel(*single_pass.rsvd_single_pass(a, k, om, philox.gaussian(2003, 1, m, 3 * (k + p)))[:3])
    assert e_l > 1.0 and e_3l < 1.0 and e_q2 < e_3l


def _dense_givens(n, i, t):
    g = np.eye(n)
    c, s = np.cos(t), np.sin(t)
    g[i, i], g[i, i + 1], g[i + 1, i], g[i + 1, i + 1] = c, s, -s, c
    return g


def test_gsrft_against_the_dense_product():
    """eq. random_Givens written out as dense matrices for n = 16: Omega = D'' Pi' G'..
    D' Pi G.. D F R, every factor built on its own."""
    n, lc = 16, 3
    seed = 5
    d, f = srft.draw(seed, n, lc)
    d1, d2, p1, p2, t1, t2 = srft.gsrft_draw(seed, n)

    def theta(p, t):
        m = np.eye(n)[p]                  # (Pi x)_k = x_p[k]
        for i in range(n - 1):
            m = m @ _dense_givens(n, i, t[i])
        return m

    dense = np.diag(d2) @ theta(p2, t2) @ np.diag(d1) @ theta(p1, t1) @ srft.omega_real(d, f)
    assert np.max(np.abs(srft.gsrft_omega_real(seed, n, lc) - dense)) <= 1e-14
    # the draws: +-1 signs, permutations, angles in [0, 2 pi)
    for x in (d1, d2):
        assert set(np.unique(x)) <= {-1.0, 1.0}
    for p in (p1, p2):
        assert sorted(p.tolist()) == list(range(n))
    assert np.all((t1 >= 0) & (t1 < 2 * np.pi)) and np.all((t2 >= 0) & (t2 < 2 * np.pi))


def test_gsrft_columns_orthogonal_and_random():
    """The left factor is orthogonal: Omega^T Omega = (n / (2 l_c)) I as for the real SRFT;
    the factors differ between seeds and are not the identity."""
    n, lc = 512, 20
    om = srft.gsrft_omega_real(11, n, lc)
    assert np.max(np.abs(om.T @ om - n / (2 * lc) * np.eye(2 * lc))) <= 1e-11
    d, f = srft.draw(11, n, lc)
    assert np.max(np.abs(om - srft.omega_real(d, f))) > 0.1
    _, _, p1, _, t1, _ = srft.gsrft_draw(11, n)
    _, _, q1, _, u1, _ = srft.gsrft_draw(12, n)
    assert not np.array_equal(p1, q1) and not np.allclose(t1, u1)
    # angles spread over the circle (a Kolmogorov-Smirnov distance far below 1)
    u = np.sort(t1 / (2 * np.pi))
    assert np.max(np.abs(u - (np.arange(1, n) - 0.5) / (n - 1))) < 0.1
