"""GPU parity of the batched randomized SVD (many small bfloat16 matrices, one plan).

Each matrix b is checked against the oracle run on the same bfloat16 values with its
own test matrix Omega_b = gaussian(seed + b, stream 0): singular values within
eps sigma_1 + 2 (the oracle's own shortfall from the true singular values), never
above the true singular values, vectors within the Wedin gap bound -- the same
acceptance as the single-matrix tensor-core path (tests/test_gpu_tc.py, _check_ritz).
"""
import os
import sys

import numpy as np
import pytest
import torch

import synth
from oracle import philox

sys.path.insert(0, os.path.dirname(__file__))
from test_gpu_tc import _check_ritz  # noqa: E402

pytestmark = pytest.mark.gpu

SHAPES = [(300, 200), (128, 64), (517, 389), (1000, 777), (2048, 1024), (129, 65), (640, 130),
          (1500, 64)]


def _make_batch(shapes, seed):
    mats, a64 = [], []
    for b, (m, n) in enumerate(shapes):
        sig = np.exp(-np.arange(min(m, n)) / 4.0)
        a, *_ = synth.lowrank(m, n, sig, seed + b)
        ab = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16)
        lda = -(-n // 8) * 8
        t = torch.zeros(m, lda, dtype=torch.bfloat16, device="cuda")
        t[:, :n] = ab.cuda()
        mats.append(t)
        a64.append(ab.float().numpy().astype(np.float64))
    return mats, a64


@pytest.mark.parametrize("k,p,q", [(16, 8, 1), (10, 6, 0), (8, 8, 2)])
def test_batched_rsvd_matches_oracle(rsvd_lib, k, p, q):
    seed = 2005
    mats, a64 = _make_batch(SHAPES, 1005)
    with rsvd_lib.BatchedPlan(SHAPES, k, p, q, seed=seed) as pl:
        U, S, V = pl.svd(mats)
        sweeps = pl.sync()
        u_all, s_all, v_all = U.cpu().double().numpy(), S.cpu().double().numpy(), V.cpu().double().numpy()
        rm, rn = pl.row_m, pl.row_n
    assert 0 < sweeps < 40
    for b, (m, n) in enumerate(SHAPES):
        om = philox.gaussian(seed + b, 0, n, k + p)
        _check_ritz(a64[b], u_all[rm[b]:rm[b + 1]], s_all[b], v_all[rn[b]:rn[b + 1]], k, p, q, om)


def test_batched_matches_single_matrix_path(rsvd_lib):
    """The batched plan and the one-matrix plan agree on a matrix they both accept."""
    m, n, k, p, q = 700, 512, 16, 8, 1
    mats, a64 = _make_batch([(m, n)], 77)
    with rsvd_lib.BatchedPlan([(m, n)], k, p, q, seed=9) as pl:
        U, S, V = pl.svd(mats)
        pl.sync()
    with rsvd_lib.Plan(m, n, k, p, q, 9, rsvd_lib.RSVD_BF16_TC) as sp:
        U1, S1, V1 = sp.svd(mats[0][:, :n].contiguous())
        torch.cuda.synchronize()
    s, s1 = S[0].cpu().double().numpy(), S1.cpu().double().numpy()
    assert np.max(np.abs(s - s1)) <= 1e-4 * s1[0]
