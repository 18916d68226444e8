"""GPU parity of the row ID (rsvd_row_id) and of Stage B by row extraction
(rsvd_svd_row_extraction, Algorithm 5.2) against oracle.row_extraction.

The pivots are integer decisions taken on float32 residual norms on the GPU and float64
ones in the oracle: they are compared exactly up to the first step at which the oracle's
two longest residuals are within 1e-3 of each other (where a rounding may decide either
way).  Beyond it several pivot sequences are correct, so the GPU's is checked for what
defines one: distinct rows, each the longest residual (to 1e-3) once the rows chosen
before it are projected out (float64, in the test), X[J] = I and Y = X Y[J].  The
shapes of the full comparison of Algorithm 5.2 are ones whose pivot choices are all
clear-cut (margins above 2e-3); there U, sigma, V are held to the float32 target 1e-5
scaled by ||X|| (the factorisation multiplies the rounding of A[J] by it); larger shapes
are held to Lemma 5.1's bound.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import metrics, mixed, philox, row_extraction, rsvd64

pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().double().cpu().numpy()


def _agree_upto(margins, thr=1e-3):
    small = np.nonzero(margins < thr)[0]
    return int(small[0]) if len(small) else len(margins)


def _greedy_valid(y, j, tol=1e-3):
    """Each pivot is the longest residual row once the earlier pivots are projected out."""
    basis = np.zeros((y.shape[1], 0))
    for i, ji in enumerate(j):
        r = y - (y @ basis) @ basis.T
        norms = np.einsum("ij,ij->i", r, r)
        if norms[ji] < (1.0 - tol) * norms.max():
            return False
        v = r[ji] / np.sqrt(norms[ji])
        v -= basis @ (basis.T @ v)
        basis = np.hstack([basis, (v / np.linalg.norm(v))[:, None]])
    return True


@pytest.mark.parametrize("m,l", [(300, 16), (2000, 48), (5000, 112), (4097, 256)])
def test_row_id_matches_oracle(rsvd_lib, m, l):
    pkg = rsvd_lib
    rng = np.random.default_rng(m + l)
    y = np.linalg.qr(rng.standard_normal((m, l)) * rng.uniform(0.1, 1.0, size=(m, 1)))[0]
    y32 = y.astype(np.float32)
    y64 = y32.astype(np.float64)
    jref, margins = row_extraction.pivot_rows(y64, l, with_margins=True)
    _, xref = row_extraction.interpolative_rows(y64)
    with pkg.Plan(m, max(l, 16), l, 0, 0, 1) as pl:
        Y = torch.tensor(y32, device="cuda")
        J = torch.zeros(l, dtype=torch.int32, device="cuda")
        X = torch.zeros(m, l, device="cuda")
        pkg.rsvd_row_id(pl.handle, Y, l, J, X, l)
        assert pkg.rsvd_sync(pl.handle) == pkg.RSVD_OK
    j, x = J.cpu().numpy().astype(np.int64), _np(X)
    t = _agree_upto(margins)
    print(f"row ID {m} x {l}: pivots agree on {np.sum(j == jref)} of {l}, clear-cut up to step {t}, "
          f"max |X| {np.abs(x).max():.2f}")
    assert np.array_equal(j[:t], jref[:t])
    assert len(set(j.tolist())) == l and j.min() >= 0 and j.max() < m
    assert _greedy_valid(y64, j)
    nx = max(1.0, np.linalg.norm(x, 2))
    assert np.max(np.abs(x[j] - np.eye(l))) <= 1e-5 * nx
    assert np.linalg.norm(y64 - x @ y64[j], 2) <= 1e-5 * nx
    if t == l:
        assert np.max(np.abs(x - xref)) <= 1e-5 * nx * max(1.0, np.abs(xref).max())


# (m, n, k, p, q, precision, matrix seed offset); the first five have clear-cut pivots
CASES = [(400, 300, 16, 0, 1, 0, 0), (600, 500, 20, 4, 1, 0, 1), (600, 504, 16, 8, 1, 1, 4),
         (800, 600, 24, 8, 1, 1, 0), (1000, 800, 12, 4, 1, 0, 0),
         (2000, 1200, 100, 12, 1, 0, 0), (3000, 2048, 64, 0, 1, 1, 0)]


@pytest.mark.parametrize("m,n,k,p,q,prec,extra", CASES)
def test_row_extraction_matches_oracle(rsvd_lib, m, n, k, p, q, prec, extra):
    pkg = rsvd_lib
    l = k + p
    sig = np.exp(-np.arange(min(m, n)) / (l / 5.0))
    a, *_ = synth.lowrank(m, n, sig, m + n + l + extra)
    tc = prec == pkg.RSVD_BF16_TC
    a_st = mixed.bf16(a.astype(np.float32)) if tc else a.astype(np.float32).astype(np.float64)
    seed = 77 + m + extra
    with pkg.Plan(m, n, k, p, q, seed, prec) as pl:
        A = torch.tensor(a_st.astype(np.float32), device="cuda")
        if tc:
            A = A.to(torch.bfloat16)
        U = torch.zeros(m, k, device="cuda")
        S = torch.zeros(k, device="cuda")
        V = torch.zeros(n, k, device="cuda")
        pkg.rsvd_svd_row_extraction(pl.handle, A, U, S, V)
        assert pkg.rsvd_sync(pl.handle) == pkg.RSVD_OK
    u, s, v = _np(U), _np(S), _np(V)
    om = philox.gaussian(seed, philox.STREAM_OMEGA, n, l)
    qref = mixed.range_finder(a_st, om, q) if tc else rsvd64.range_finder(a_st, om, q)
    uf, sf, vf, jref, xref = row_extraction.svd_row_extraction(a_st, qref)
    _, margins = row_extraction.pivot_rows(qref, l, with_margins=True)
    t = _agree_upto(margins, 2e-3)
    nx = max(1.0, np.linalg.norm(xref, 2))
    eps_q = metrics.projection_error(a_st, qref)
    err = np.linalg.norm(a_st - (u * s) @ v.T, 2)
    tail = sf[k] if k < l else 0.0
    print(f"row extraction {m}x{n} l={l} q={q} prec={prec}: clear-cut pivots {t}/{l}, ||X|| {nx:.2f}, "
          f"error {err:.3e} (basis {eps_q:.3e}), max |dsigma| / sigma_1 {np.max(np.abs(s - sf[:k])) / sf[0]:.2e}")
    assert metrics.orthonormality(u) <= 2e-5 and metrics.orthonormality(v) <= 2e-5
    assert err <= (1.0 + nx) * eps_q * 1.05 + tail + 1e-5 * nx * sf[0]
    if t == l:
        eps = 1e-5 * nx
        assert np.max(np.abs(s - sf[:k])) <= eps * sf[0]
        bound = metrics.gap_bound(sf[:k], eps, c=1.0, s_next=tail if k < l else None) + eps
        d = np.sign(np.sum(u * uf[:, :k], axis=0))
        d[d == 0] = 1.0
        assert np.all(np.linalg.norm(u * d - uf[:, :k], axis=0) <= bound)
        assert np.all(np.linalg.norm(v * d - vf[:, :k], axis=0) <= bound)
    else:
        assert np.max(np.abs(s - sf[:k])) <= 2.0 * (1.0 + nx) * eps_q
