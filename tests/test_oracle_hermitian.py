"""Pins of oracle.hermitian (Algorithms 5.3 and 5.5; CPU only).

* Exact recovery: for a symmetric A of rank r <= l the basis from Stage A spans its range,
  and both algorithms return its eigenpairs to 1e-12.
* Algorithm 5.3 keeps the error within twice the range finder's (the 2 eps bound of
  Section 5.3): ||A - U Lambda U^T|| <= 2 ||A - Q Q^T A|| (with k = l).
* Algorithm 5.5 (psd A): ||A - F F^T|| <= ||A - Q Q^T A|| (the Nystrom bound the section
  quotes), and on a decaying spectrum it is markedly smaller; Lambda >= 0.
* Both: U orthonormal; eigenvalues sorted by decreasing |lambda|; an indefinite A keeps
  the signs of its eigenvalues in Algorithm 5.3.
"""
import numpy as np

import synth
from oracle import hermitian, metrics, rsvd64


def _sym(n, lam, seed):
    q = synth.haar(np.random.default_rng(seed), n, len(lam))
    return (q * lam) @ q.T


def test_exact_recovery():
    n, k, p = 300, 8, 6
    lam = np.array([5.0, -4.0, 3.0, 2.5, -1.0, 0.5])
    a = _sym(n, lam, 1)
    om = np.random.default_rng(2).standard_normal((n, k + p))
    qmat = rsvd64.range_finder(a, om, 1)
    u, l_d = hermitian.eig_direct(a, qmat, 6)
    assert np.allclose(l_d, lam[np.argsort(-np.abs(lam), kind="stable")], atol=1e-12)
    assert np.linalg.norm(a - (u * l_d) @ u.T, 2) <= 1e-12 * 5.0
    apsd = _sym(n, np.abs(lam), 1)
    qp = rsvd64.range_finder(apsd, om, 1)
    u2, l_n, f = hermitian.nystrom(apsd + 1e-13 * np.eye(n), qp, 6)
    assert np.allclose(l_n, np.sort(np.abs(lam))[::-1], atol=1e-10)


def test_direct_within_twice_the_range_finder_error():
    n, k, p = 400, 20, 10
    lam = np.exp(-np.arange(n) / 6.0) * np.where(np.arange(n) % 3 == 1, -1.0, 1.0)
    a = _sym(n, lam, 3)
    for seed in range(5):
        om = np.random.default_rng(10 + seed).standard_normal((n, k + p))
        qmat = rsvd64.range_finder(a, om, 0)
        u, lam_d = hermitian.eig_direct(a, qmat, k + p)
        e_range = metrics.projection_error(a, qmat)
        e_eig = np.linalg.norm(a - (u * lam_d) @ u.T, 2)
        assert e_eig <= 2.0 * e_range * (1 + 1e-10)
        assert metrics.orthonormality(u) <= 1e-13
        assert np.all(np.diff(np.abs(lam_d)) <= 1e-15)
        assert np.any(lam_d < 0)                     # the indefinite spectrum keeps its signs


def test_nystrom_never_worse_than_the_range_finder():
    n, k, p = 400, 20, 10
    lam = np.exp(-np.arange(n) / 6.0)
    a = _sym(n, lam, 4)
    better = 0
    for seed in range(5):
        om = np.random.default_rng(20 + seed).standard_normal((n, k + p))
        qmat = rsvd64.range_finder(a, om, 0)
        u, lam_n, f = hermitian.nystrom(a, qmat, k + p)
        e_range = metrics.projection_error(a, qmat)
        e_ny = np.linalg.norm(a - f @ f.T, 2)
        assert e_ny <= e_range * (1 + 1e-8)
        assert np.all(lam_n >= 0) and metrics.orthonormality(u) <= 1e-13
        # U Lambda U^T is F F^T
        assert np.linalg.norm((u * lam_n) @ u.T - f @ f.T, 2) <= 1e-12
        better += e_ny < 0.6 * e_range             # about 0.45 here: one free subspace step
    assert better >= 4
