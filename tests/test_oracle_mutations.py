"""Plant plausible mistakes in the oracle and check that its pins reject them (CPU only).

Each mutation is applied with monkeypatch to the oracle module, then the pin
that should notice it is re-run and must fail.
"""
import numpy as np
import pytest

import tests.test_oracle_pins as pins
from oracle import philox, rsvd64, single_pass, srft


def _fails(fn, *args):
    with pytest.raises((AssertionError, ValueError)):
        fn(*args)


def test_philox_swapped_halves_is_caught(monkeypatch):
    orig = philox.philox4x32_10

    def bad(counter, key):
        out = orig(counter, key)
        return out[:, [1, 0, 2, 3]]

    monkeypatch.setattr(philox, "philox4x32_10", bad)
    _fails(pins.test_philox_known_answers)


def test_box_muller_wrong_branch_is_caught(monkeypatch):
    def bad(seed, stream, rows, cols):
        groups = (cols + 3) // 4
        u = philox.bits_to_uniform(philox.raw_words(seed, stream, rows, groups))
        r = np.sqrt(-2.0 * np.log(u[..., 0]))
        z = np.stack([r * np.cos(2 * np.pi * u[..., 1])] * 4, axis=-1)   # cos for every output
        return z.reshape(rows, groups * 4)[:, :cols]

    monkeypatch.setattr(philox, "gaussian", bad)
    _fails(pins.test_gaussian_layout_and_moments)


def test_dropped_power_step_is_caught(monkeypatch):
    orig = rsvd64.range_finder

    def bad(a, omega, q=0, keep_steps=False):
        return orig(a, omega, 0, keep_steps) if not keep_steps else orig(a, omega, 0, True)

    monkeypatch.setattr(rsvd64, "range_finder", bad)
    _fails(pins.test_power_spectrum_and_algorithm_4_3_equivalence)


def test_missing_qr_sign_fix_is_caught(monkeypatch):
    def bad(y):
        q, r = np.linalg.qr(y)
        return -q, -r

    monkeypatch.setattr(rsvd64, "qr_pos", bad)
    _fails(pins.test_qr_pos)


def test_wrong_truncation_is_caught(monkeypatch):
    monkeypatch.setattr(rsvd64, "truncate", lambda u, s, v, k: (u[:, -k:], s[-k:], v[:, -k:]))
    _fails(pins.test_truncation_theorem_9_3_and_no_degradation)


def test_transposed_stage_b_is_caught(monkeypatch):
    def bad(a, qmat):
        b = qmat.T @ a
        ut, s, vt = np.linalg.svd(b, full_matrices=False)
        return qmat @ ut, s, vt          # V returned untransposed
    monkeypatch.setattr(rsvd64, "direct_svd", bad)
    _fails(pins.test_truncation_theorem_9_3_and_no_degradation)


def test_srft_missing_scale_is_caught(monkeypatch):
    orig = srft.omega_complex
    monkeypatch.setattr(srft, "omega_complex", lambda d, f: orig(d, f) / np.sqrt(d.shape[0] / f.shape[0]))
    _fails(pins.test_srft_structure)


def test_sylvester_sign_error_is_caught(monkeypatch):
    def bad(x1, c1, x2, c2):
        p = x2 @ x2.T
        s = x1 @ x1.T
        rhs = c1 @ x1.T - x2 @ c2.T
        lp, up = np.linalg.eigh(p)
        ls, us = np.linalg.eigh(s)
        return up @ ((up.T @ rhs @ us) / (lp[:, None] + ls[None, :])) @ us.T

    monkeypatch.setattr(single_pass, "min_residual", bad)
    _fails(pins.test_single_pass_solver_matches_bruteforce)


def test_dropped_lo_half_is_caught(monkeypatch):
    import tests.test_oracle_mixed as mpins
    from oracle import mixed

    monkeypatch.setattr(mixed, "split", lambda x: mixed.bf16(x))
    _fails(mpins.test_exact_rank_recovery_limited_by_the_split_basis)


def test_rounded_basis_in_the_lift_is_caught(monkeypatch):
    import tests.test_oracle_mixed as mpins
    from oracle import mixed

    orig = mixed.range_finder
    monkeypatch.setattr(mixed, "range_finder", lambda *a, **kw: mixed.bf16(orig(*a, **kw)))
    _fails(mpins.test_lift_uses_the_float64_basis)


def test_unrounded_test_matrix_is_caught(monkeypatch):
    import tests.test_oracle_mixed as mpins
    from oracle import mixed

    orig = mixed.range_finder
    monkeypatch.setattr(mixed, "range_finder",
                        lambda a, om, q, operand=None: orig(a, om, q, operand=lambda x: x))
    _fails(mpins.test_first_sample_uses_the_rounded_test_matrix)


def test_dropped_power_step_in_the_gradient_is_caught(monkeypatch):
    from oracle import grad

    orig = grad._rsvd_torch
    monkeypatch.setattr(grad, "_rsvd_torch", lambda at, om, k, q: orig(at, om, k, 0))
    _fails(pins.test_cotangent_gradient_autograd_vs_finite_differences)


def test_adaptive_without_the_second_reprojection_is_caught(monkeypatch):
    import tests.test_oracle_adaptive as apins
    from oracle import adaptive

    monkeypatch.setattr(adaptive, "orth_block",
                        lambda q, y: adaptive.qr_pos(adaptive.project_out(q, y))[0])
    _fails(apins.test_exact_rank_recovery)


def test_adaptive_threshold_without_the_estimate_constant_is_caught(monkeypatch):
    import tests.test_oracle_adaptive as apins
    from oracle import adaptive

    monkeypatch.setattr(adaptive, "THRESHOLD_FACTOR", 1.0 / 100.0)   # stops far too early
    _fails(apins.test_tolerance_is_met_and_the_basis_is_economical, 1e-4, 8)


def test_row_pivoting_on_the_shortest_row_is_caught(monkeypatch):
    import tests.test_oracle_row_extraction as rpins
    from oracle import row_extraction

    def bad(y, count):
        r = np.array(y, dtype=np.float64, copy=True)
        chosen = []
        for _ in range(count):
            norms = np.einsum("ij,ij->i", r, r)
            norms[chosen] = np.inf
            j = int(np.argmin(norms))
            chosen.append(j)
            v = r[j] / np.linalg.norm(r[j])
            r -= np.outer(r @ v, v)
        return np.array(chosen)

    monkeypatch.setattr(row_extraction, "pivot_rows", bad)
    _fails(rpins.test_pivots_match_lapack_column_pivoted_qr)


def test_untransposed_r_in_row_extraction_is_caught(monkeypatch):
    import tests.test_oracle_row_extraction as rpins
    from oracle import row_extraction

    def bad(a, qmat):
        jset, x = row_extraction.interpolative_rows(qmat)
        w, r = row_extraction.qr_pos(a[jset].T)
        u, s, vt_t = np.linalg.svd(x @ r, full_matrices=False)     # R where R^T belongs
        return u, s, w @ vt_t.T, jset, x

    monkeypatch.setattr(row_extraction, "svd_row_extraction", bad)
    _fails(rpins.test_lemma_5_1_identity_and_bound)


def test_givens_chain_in_the_wrong_order_is_caught(monkeypatch):
    def bad(theta, x):
        y = np.array(x, dtype=np.float64, copy=True)
        for i in range(len(theta)):                      # leftmost rotation first
            c, s = np.cos(theta[i]), np.sin(theta[i])
            yi, yj = y[i].copy(), y[i + 1].copy()
            y[i] = c * yi + s * yj
            y[i + 1] = -s * yi + c * yj
        return y

    monkeypatch.setattr(srft, "givens_chain", bad)
    _fails(pins.test_gsrft_against_the_dense_product)


def test_a_last_ignored_is_caught(monkeypatch):
    """range_finder that lets every product see a_stored (a_last dropped) must fail the pin
    of the residual-in-the-final-bases reading."""
    import tests.test_oracle_mixed as mpins
    from oracle import mixed

    orig = mixed.range_finder
    monkeypatch.setattr(mixed, "range_finder",
                        lambda a_stored, omega, q, operand=None, a_last=None: orig(a_stored, omega, q, operand))
    _fails(mpins.test_last_product_sees_a_last)


def test_a_last_in_every_product_is_caught(monkeypatch):
    """range_finder that uses a_last in every product of Stage A (the early ones too)."""
    import tests.test_oracle_mixed as mpins
    from oracle import mixed

    orig = mixed.range_finder

    def bad(a_stored, omega, q, operand=None, a_last=None):
        return orig(a_stored if a_last is None else a_last, omega, q, operand)

    monkeypatch.setattr(mixed, "range_finder", bad)
    _fails(mpins.test_last_product_sees_a_last)
