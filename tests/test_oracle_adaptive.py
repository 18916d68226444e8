"""Pins of oracle.adaptive (blocked Algorithm 4.2, the fixed-precision range finder; CPU only).

* Lemma 4.1, the posterior estimate the stopping rule rests on: for a fixed B and r
  Gaussian vectors, ||B|| <= alpha sqrt(2/pi) max_i ||B w_i|| fails with probability at
  most alpha^-r -- checked by frequency over many draws, with an alpha small enough that
  the bound is nearly attained (so a wrong constant shows).
* The guarantee of Algorithm 4.2: ||(I - Q Q^T) A|| <= eps on every seed and tolerance tried.
* Exact-rank inputs: the basis captures A exactly and stops at the first whole block past
  the rank.
* Economy: the basis is no wider than the singular values above the threshold need plus a
  block or two (a stopping rule that is far too strict shows up here).
* Orthonormality to 1e-13 even when the consumed samples are tiny (the reprojection of
  step 7).
"""
import numpy as np
import pytest

import synth
from oracle import adaptive, metrics


def test_lemma_4_1_failure_probability():
    rng = np.random.default_rng(0)
    a, *_ = synth.lowrank(60, 40, np.array([3.0, 2.0, 1.0, 0.5, 0.1]), 1)
    nb = np.linalg.norm(a, 2)
    alpha, r, trials = 1.5, 3, 4000
    fails = 0
    for _ in range(trials):
        w = rng.standard_normal((40, r))
        est = alpha * np.sqrt(2.0 / np.pi) * np.max(np.linalg.norm(a @ w, axis=0))
        fails += est < nb
    rate = fails / trials
    assert rate <= alpha ** -r + 3 * np.sqrt(alpha ** -r / trials)
    # the bound is not vacuous here: with half the constant it fails far more often
    fails2 = 0
    for _ in range(trials):
        w = rng.standard_normal((40, r))
        fails2 += 0.5 * alpha * np.sqrt(2.0 / np.pi) * np.max(np.linalg.norm(a @ w, axis=0)) < nb
    assert fails2 / trials > 2 * alpha ** -r


@pytest.mark.parametrize("eps", [1e-2, 1e-4, 1e-7])
@pytest.mark.parametrize("block", [4, 8])
def test_tolerance_is_met_and_the_basis_is_economical(eps, block):
    m, n = 220, 160
    sig = np.exp(-np.arange(n) / 8.0)
    a, *_ = synth.lowrank(m, n, sig, 3)
    cap = 152                                         # room for the 1e-7 basis (about 130)
    for seed in range(8):
        om = np.random.default_rng(100 + seed).standard_normal((n, cap + block))
        q, est = adaptive.adaptive_range_finder(a, eps, om, block, cap)
        err = metrics.projection_error(a, q)
        assert err <= eps
        assert metrics.orthonormality(q) <= 1e-13
        need = int(np.sum(sig > eps / 1e3))            # far below the threshold
        assert q.shape[1] <= need + 2 * block
        assert q.shape[1] % block == 0


def test_exact_rank_recovery():
    m, n, r, block = 300, 200, 20, 16
    a, *_ = synth.lowrank(m, n, np.linspace(2.0, 0.5, r), 7)
    om = np.random.default_rng(1).standard_normal((n, 96 + block))
    q, est = adaptive.adaptive_range_finder(a, 1e-10, om, block, 96)
    assert q.shape[1] == 32                          # two blocks hold the 20 directions
    assert metrics.projection_error(a, q) <= 1e-12 * np.linalg.norm(a, 2)
    assert est <= 1e-12


def test_orthonormal_when_the_samples_are_tiny():
    m, n, block = 200, 120, 8
    sig = 10.0 ** (-np.arange(n) / 3.0)
    a, *_ = synth.lowrank(m, n, sig, 11)
    om = np.random.default_rng(2).standard_normal((n, 96 + block))
    q, _ = adaptive.adaptive_range_finder(a, 1e-13, om, block, 96)
    assert q.shape[1] >= 40
    assert metrics.orthonormality(q) <= 1e-13
