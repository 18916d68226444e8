"""Pins of oracle.mixed, the float64 model of the tensor-core precision pattern (CPU only).

The pattern (Algorithm 4.4 + Algorithm 5.1 with bfloat16 operands in Stage A and a
hi + lo basis in B^T = A^T Q) has no printed worked example; it is pinned by:
  * the bfloat16 rounding against its definition (hand-computed ties and spacings)
    and against torch's float32 -> bfloat16 conversion, a library routine;
  * exact-rank recovery: the rounded operands do not change the range of a rank-r
    matrix, so only the 16-bit basis of the final product limits the error
    (2^-16 ||A||; a dropped lo half would leave about 2^-8);
  * orthonormality of U to float64 precision (the lift must use Q, not its rounding);
  * identity roundings reproduce the pinned oracle rsvd64.rsvd exactly;
  * the matched-error reading: hi + lo in every product keeps ||A - U S V^T||_F
    within 1e-4 of the float64 path's, a bfloat16 Stage A does not.
"""
import numpy as np
import pytest

import synth
from oracle import metrics, mixed, rsvd64


def test_bf16_rounding_definition():
    f = mixed.bf16
    # representable values are fixed points (8 significant bits)
    for x in (0.0, 1.0, -2.5, 1.0 + 2.0 ** -7, 255.0, 2.0 ** -126, 3.0 * 2.0 ** -133):
        assert f(x) == x
    # ties go to the even neighbour; spacing 2^-7 in [1, 2)
    assert f(1.0 + 2.0 ** -8) == 1.0
    assert f(1.0 + 3.0 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert f(-(1.0 + 3.0 * 2.0 ** -8)) == -(1.0 + 2.0 ** -6)
    assert f(1.0 + 2.0 ** -8 + 2.0 ** -30) == 1.0 + 2.0 ** -7     # above the tie: up
    assert f(np.pi) == 3.140625
    # spacing 2^-133 below the smallest normal 2^-126
    assert f(2.0 ** -133 * 1.4) == 2.0 ** -133 and f(2.0 ** -133 * 0.4) == 0.0
    x = np.random.default_rng(0).standard_normal(10000) * 10.0 ** np.random.default_rng(1).uniform(-20, 20, 10000)
    r = f(x)
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x))      # unit roundoff of 8 bits
    assert np.array_equal(f(r), r)


def test_bf16_matches_library_conversion():
    import torch

    rng = np.random.default_rng(3)
    x = (rng.standard_normal(200000) * 10.0 ** rng.uniform(-30, 30, 200000)).astype(np.float32)
    lib = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mixed.bf16(x.astype(np.float64)), lib)


def test_split_carries_sixteen_bits():
    x = np.random.default_rng(4).standard_normal(10000)
    s = mixed.split(x)
    assert np.all(np.abs(s - x) <= 2.0 ** -16 * np.abs(x))
    assert np.all(mixed.bf16(s - mixed.bf16(x)) == s - mixed.bf16(x))   # lo is a bfloat16 value


def test_exact_rank_recovery_limited_by_the_split_basis():
    m, n, r, k, p, q = 300, 200, 6, 10, 4, 1
    a, *_ = synth.lowrank(m, n, np.array([3.0, 2.0, 1.5, 1.0, 0.5, 0.25]), 11)
    omega = np.random.default_rng(2).standard_normal((n, k + p))
    u, s, v, qmat = mixed.rsvd(a, k, p, q, omega)
    err = np.linalg.norm(a - (u * s) @ v.T, 2) / np.linalg.norm(a, 2)
    assert err <= 2.0 ** -16 and err > 1e-12          # the 16-bit basis of B^T = A^T Q shows
    assert metrics.projection_error(a, qmat) <= 1e-12 * np.linalg.norm(a, 2)   # Stage A exact
    np.testing.assert_allclose(s[:r], [3.0, 2.0, 1.5, 1.0, 0.5, 0.25], rtol=2.0 ** -15)
    # with Q itself in the final product the recovery is exact
    u2, s2, v2, _ = mixed.rsvd(a, k, p, q, omega, final_basis=lambda x: x)
    assert np.linalg.norm(a - (u2 * s2) @ v2.T, 2) <= 1e-12 * np.linalg.norm(a, 2)


def test_lift_uses_the_float64_basis():
    a, *_ = synth.lowrank(400, 300, synth.spectrum_exp(300, 5.0), 5)
    omega = np.random.default_rng(6).standard_normal((300, 24))
    u, s, v, _ = mixed.rsvd(a, 16, 8, 1, omega)
    assert metrics.orthonormality(u) <= 1e-13
    assert metrics.orthonormality(v) <= 1e-13


def test_identity_roundings_reproduce_rsvd64():
    a, *_ = synth.lowrank(250, 180, synth.spectrum_exp(180, 8.0), 9)
    omega = np.random.default_rng(8).standard_normal((180, 20))
    ident = lambda x: x  # noqa: E731
    u, s, v, qm = mixed.rsvd(a, 12, 8, 2, omega, operand=ident, final_basis=ident)
    u0, s0, v0, q0 = rsvd64.rsvd(a, 12, 8, 2, omega)
    assert np.allclose(s, s0, rtol=0, atol=1e-13)
    assert np.allclose(np.abs(np.sum(u * u0, axis=0)), 1.0, atol=1e-10)
    assert np.allclose(qm, q0, atol=1e-12)


@pytest.mark.parametrize("seed", [77, 78])
def test_residual_in_every_product_reaches_matched_error(seed):
    m = n = 2048
    k, p, q = 100, 10, 1
    a, *_ = synth.lowrank(m, n, synth.spectrum_power(n, 1.5), seed)
    a = a.astype(np.float32).astype(np.float64)
    omega = np.random.default_rng(seed).standard_normal((n, k + p))
    e_ref = metrics.fro_error(a, *rsvd64.rsvd(a, k, p, q, omega)[:3])
    hi = mixed.bf16(a)
    hl = mixed.split(a)
    every = metrics.fro_error(a, *mixed.rsvd(hl, k, p, q, omega)[:3])
    bf_stage_a = metrics.fro_error(a, *mixed.rsvd(hi, k, p, q, omega, a_final=hl)[:3])
    assert abs(every - e_ref) / e_ref <= 1e-4
    assert (bf_stage_a - e_ref) / e_ref > 5e-4


def test_first_sample_uses_the_rounded_test_matrix():
    """Algorithm 4.4 step 2 under the pattern: Q0 spans A bf16(Omega), whose columns are
    exact in float64 for a small-integer A (no accumulation error to hide a missing
    rounding), and differs from the span of A Omega."""
    rng = np.random.default_rng(12)
    a = rng.integers(-3, 4, size=(60, 40)).astype(np.float64)
    omega = rng.standard_normal((40, 8))
    q0 = mixed.range_finder(a, omega, 0)
    y = a @ mixed.bf16(omega)
    assert np.linalg.norm(y - q0 @ (q0.T @ y)) <= 1e-12 * np.linalg.norm(y)
    y_unrounded = a @ omega
    assert np.linalg.norm(y_unrounded - q0 @ (q0.T @ y_unrounded)) > 1e-6 * np.linalg.norm(y_unrounded)


def test_last_product_sees_a_last():
    """a_last enters the last product of Stage A only: with q = 0 it is the only product;
    with q = 1 and a_last zero outside a set of rows, the final basis is zero outside those
    rows too, while the intermediate basis still comes from a_stored (so Q differs from the
    basis with that restricted matrix in every product)."""
    rng = np.random.default_rng(21)
    a = rng.standard_normal((80, 50))
    x = rng.standard_normal((80, 50))
    omega = rng.standard_normal((50, 6))
    assert np.array_equal(mixed.range_finder(x, omega, 0, a_last=a), mixed.range_finder(a, omega, 0))
    rows = np.arange(80) % 3 == 0
    a_r = np.where(rows[:, None], a, 0.0)
    qm = mixed.range_finder(a, omega, 1, a_last=a_r)
    assert np.max(np.abs(qm[~rows])) <= 1e-15
    assert metrics.orthonormality(qm) <= 1e-13
    q_all = mixed.range_finder(a_r, omega, 1)
    assert np.linalg.norm(qm @ qm.T - q_all @ q_all.T) > 1e-3


@pytest.mark.parametrize("seed", [77, 78])
def test_residual_in_the_final_bases_sits_between(seed):
    """The residual lo in the products that make the final bases (the last of Stage A and
    B^T = A^T Q) and hi alone in the earlier power-iteration product: the error of the
    hi-only product is only partly washed out by the one product after it (q = 1), so the
    excess lands between the two patterns above -- at most half that of hi alone in all of
    Stage A, but above the 1e-4 of the residual in every product on some draws (6e-4 for
    seed 78)."""
    m = n = 2048
    k, p, q = 100, 10, 1
    a, *_ = synth.lowrank(m, n, synth.spectrum_power(n, 1.5), seed)
    a = a.astype(np.float32).astype(np.float64)
    omega = np.random.default_rng(seed).standard_normal((n, k + p))
    e_ref = metrics.fro_error(a, *rsvd64.rsvd(a, k, p, q, omega)[:3])
    hi = mixed.bf16(a)
    hl = mixed.split(a)
    final_bases = metrics.fro_error(a, *mixed.rsvd(hi, k, p, q, omega, a_final=hl, a_last=hl)[:3])
    stage_a_hi = metrics.fro_error(a, *mixed.rsvd(hi, k, p, q, omega, a_final=hl)[:3])
    assert (final_bases - e_ref) / e_ref <= 0.5 * (stage_a_hi - e_ref) / e_ref
    assert (final_bases - e_ref) / e_ref <= 1e-3
