"""Pins of oracle.row_extraction (Algorithm 5.2 and the row ID it rests on; CPU only).

* A 4 x 2 ID worked by hand (tests/golden/id_rows_4x2.txt): the pivots and X.
* The pivot order is that of LAPACK's column-pivoted QR (xGEQP3, Businger--Golub with
  norm downdating) applied to Y^T, on inputs whose pivot choices are clear-cut.
* The ID itself: X[J] = I and Y = X Y[J] to 1e-13.
* Lemma 5.1: U Sigma V^T = X A[J, :] (the identity its proof starts from) to 1e-12, and
  ||A - U Sigma V^T|| <= (1 + ||X||) ||A - Q Q^T A|| (its bound before the entries of X
  are bounded), on every seed.
* Exact rank: for rank(A) <= l the factorisation is exact; U, V orthonormal, sigma sorted.
"""
import os

import numpy as np
import scipy.linalg

import synth
from oracle import metrics, row_extraction, rsvd64

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "id_rows_4x2.txt")) if ln.strip() and ln[0] != "#"]
    y = np.array(rows[0:4], dtype=float)
    jset = np.array(rows[4], dtype=int)
    x = np.array(rows[5:9], dtype=float)
    return y, jset, x


def test_hand_worked_id():
    y, jset, x = _read_golden()
    j2, x2 = row_extraction.interpolative_rows(y)
    assert list(j2) == list(jset)
    assert np.allclose(x2, x, atol=1e-15)


def test_pivots_match_lapack_column_pivoted_qr():
    for seed in range(6):
        rng = np.random.default_rng(seed)
        y = rng.standard_normal((300, 12)) * np.exp(-np.arange(12) / 3.0)
        y = y * rng.uniform(0.2, 1.0, size=(300, 1))          # uneven row norms
        jset = row_extraction.pivot_rows(y, 12)
        _, _, piv = scipy.linalg.qr(y.T, pivoting=True, mode="economic")
        assert list(jset) == list(piv[:12])


def test_id_identity():
    rng = np.random.default_rng(3)
    q, _ = np.linalg.qr(rng.standard_normal((500, 20)))
    jset, x = row_extraction.interpolative_rows(q)
    assert len(set(jset.tolist())) == 20
    assert np.array_equal(x[jset], np.eye(20))
    assert np.max(np.abs(q - x @ q[jset])) <= 1e-13


def test_lemma_5_1_identity_and_bound():
    m, n, k, p = 400, 300, 20, 10
    sig = np.exp(-np.arange(n) / 6.0)
    a, *_ = synth.lowrank(m, n, sig, 5)
    for seed in range(6):
        om = np.random.default_rng(40 + seed).standard_normal((n, k + p))
        qmat = rsvd64.range_finder(a, om, 0)
        u, s, v, jset, x = row_extraction.svd_row_extraction(a, qmat)
        assert np.max(np.abs((u * s) @ v.T - x @ a[jset])) <= 1e-12
        eps = metrics.projection_error(a, qmat)
        err = np.linalg.norm(a - (u * s) @ v.T, 2)
        assert err <= (1.0 + np.linalg.norm(x, 2)) * eps * (1 + 1e-9)
        assert err >= eps * (1 - 1e-9)                      # never better than the basis
        assert metrics.orthonormality(u) <= 1e-12 and metrics.orthonormality(v) <= 1e-12
        assert np.all(np.diff(s) <= 0)


def test_exact_rank_recovery():
    m, n, r, l = 250, 180, 12, 16
    a, *_ = synth.lowrank(m, n, np.linspace(3.0, 1.0, r), 9)
    om = np.random.default_rng(2).standard_normal((n, l))
    qmat = rsvd64.range_finder(a, om, 0)
    u, s, v, _, _ = row_extraction.svd_row_extraction(a, qmat)
    assert np.linalg.norm(a - (u * s) @ v.T, 2) <= 1e-12 * 3.0
    assert np.allclose(s[:r], np.linspace(3.0, 1.0, r), atol=1e-12)
