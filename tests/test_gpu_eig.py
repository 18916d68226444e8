"""GPU parity of the Hermitian Stage B (rsvd_eig: Algorithms 5.3 and 5.5) against
oracle.hermitian.

A = V diag(lambda) V^T (Haar V), stored as float32 (plain path) or bfloat16 (tensor-core
path); rounding keeps it exactly symmetric.  Omega is the Philox draw of the plan's seed
(the same one rsvd_svd takes).  The reference basis is Algorithm 4.4 in float64 on the
stored A: oracle.rsvd64.range_finder for the plain path, oracle.mixed.range_finder (the
bfloat16 operands of the Stage A products) for the tensor-core path, whose B1 = A Q also
takes the basis as a hi + lo pair (operand = mixed.split).  Then oracle.hermitian.

Tolerances, the float32 targets of the library: |lambda_j - lambda_j^ref| <= 1e-5
|lambda_1|; eigenvectors, after sign alignment, ||u_j - u_j^ref|| <= 1e-5 |lambda_1| /
gap_j + 1e-5 with gap_j the distance of |lambda_j| to its neighbours' magnitudes (a
lower bound on the distance to the other eigenvalues, so the bound is on the safe side).
"""
import numpy as np
import pytest
import torch

import synth
from oracle import hermitian, metrics, mixed, philox, rsvd64

pytestmark = pytest.mark.gpu

EPS = 1e-5


def _np(t):
    return t.detach().double().cpu().numpy()


def _sym(n, lam, seed):
    v = synth.haar(np.random.default_rng(seed), n, len(lam))
    return (v * lam) @ v.T


def _run(pkg, a_stored, k, p, q, seed, prec, method):
    n = a_stored.shape[0]
    dt = torch.bfloat16 if prec == pkg.RSVD_BF16_TC else torch.float32
    with pkg.Plan(n, n, k, p, q, seed, prec) as pl:
        A = torch.tensor(a_stored.astype(np.float32), device="cuda").to(dt)
        U = torch.zeros(n, k, device="cuda")
        L = torch.zeros(k, device="cuda")
        pkg.rsvd_eig(pl.handle, A, method, U, L)
        assert pkg.rsvd_sync(pl.handle) == pkg.RSVD_OK
    return _np(U), _np(L)


CASES = [(1500, 24, 8, 1, 0), (2000, 100, 20, 1, 0), (1504, 24, 8, 1, 1), (2048, 100, 20, 0, 1)]


@pytest.mark.parametrize("n,k,p,q,prec", CASES)
@pytest.mark.parametrize("method", [0, 1])
def test_eig_matches_oracle(rsvd_lib, n, k, p, q, prec, method):
    pkg = rsvd_lib
    i = np.arange(n)
    lam = np.exp(-i / ((k + p) / 4.0))    # lambda_l / lambda_1 = e^-4: B = C^T C stays
                                          # well conditioned for the float32 Cholesky
    if method == pkg.RSVD_EIG_DIRECT:
        lam = lam * np.where(i % 3 == 1, -1.0, 1.0)      # indefinite; magnitudes distinct
    a = _sym(n, lam, n + k)
    tc = prec == pkg.RSVD_BF16_TC
    a_st = mixed.bf16(a.astype(np.float32)) if tc else a.astype(np.float32).astype(np.float64)
    seed = 31 + n
    u, lv = _run(pkg, a_st, k, p, q, seed, prec, method)
    om = philox.gaussian(seed, philox.STREAM_OMEGA, n, k + p)
    qref = mixed.range_finder(a_st, om, q) if tc else rsvd64.range_finder(a_st, om, q)
    op = mixed.split if tc else None
    if method == pkg.RSVD_EIG_DIRECT:
        ufull, lfull = hermitian.eig_direct(a_st, qref, k + p, operand=op)
    else:
        ufull, lfull, _ = hermitian.nystrom(a_st, qref, k + p, operand=op)
    ur, lr = ufull[:, :k], lfull[:k]
    print(f"eig n={n} k={k} q={q} prec={prec} method={method}: max |dlambda| / |lambda_1| = "
          f"{np.max(np.abs(lv - lr)) / abs(lr[0]):.2e}")
    assert np.max(np.abs(lv - lr)) <= EPS * abs(lr[0])
    if method == pkg.RSVD_EIG_NYSTROM:
        assert np.all(lv >= 0)
    mag = np.abs(lr)
    bound = metrics.gap_bound(mag, EPS, c=1.0, s_next=abs(lfull[k])) + EPS
    d = np.sign(np.sum(u * ur, axis=0))
    d[d == 0] = 1.0
    du = np.linalg.norm(u * d - ur, axis=0)
    assert np.all(du <= bound), (du / bound).max()
    assert metrics.orthonormality(u) <= 2e-5


def test_eig_rejects_a_rectangular_plan(rsvd_lib):
    pkg = rsvd_lib
    with pkg.Plan(600, 500, 10, 6, 0, 1) as pl:
        A = torch.zeros(600, 500, device="cuda")
        U = torch.zeros(600, 10, device="cuda")
        L = torch.zeros(10, device="cuda")
        with pytest.raises(pkg.RsvdError):
            pkg.rsvd_eig(pl.handle, A, pkg.RSVD_EIG_DIRECT, U, L)
