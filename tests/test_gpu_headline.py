"""The timed configuration at full size against the float64 oracle.

16384 x 16384 A = U diag(j^-1.5) V^T (Haar U, V), k = 100, p = 10, q = 1, A stored as
bfloat16 hi + lo and read in full by every pass (residual_passes = 1), exactly as the
bench times it.

Two references, both float64 with the same Omega:
  * oracle.mixed.rsvd on the stored hi + lo -- Algorithm 4.4 + 5.1 with the roundings
    the tensor-core form makes by design (bfloat16 operands of the Stage A products, the
    hi + lo basis in B^T = A^T Q).  What remains between it and the GPU is float32
    arithmetic: the tensor cores' float32 accumulation, the float32 Cholesky-QR and
    Jacobi steps, and the operands the GPU rounds from its float32 bases (a rounding
    can land on the other side of a bfloat16 tie).  The stated float32 targets apply:
    |sigma_j - sigma_j^ref| <= 1e-5 sigma_1, and for the singular vectors, after sign
    alignment, ||x_j - x_j^ref|| <= 1e-5 sigma_1 / gap_j + 1e-5 (Wedin's bound for a
    perturbation of size 1e-5 sigma_1; gap_j the distance of sigma_j to its neighbours,
    sigma_{k+1} for the last).
  * oracle.rsvd64.rsvd on the float32 A -- the method with no rounding at all.  The
    roundings by design move sigma by |sigma^mixed - sigma^plain| (computed here), so
    the GPU must stay within that plus the float32 target; and its reconstruction error
    ||A - U S V^T||_F must exceed the float64 method's by at most 1e-4 relative (the
    matched-error target).
"""
import numpy as np
import pytest
import torch

import synth
from oracle import metrics, mixed, philox, rsvd64

pytestmark = pytest.mark.gpu

EPS = 1e-5


def _np(t):
    return t.detach().double().cpu().numpy()


def _vec_dist(x, xr):
    d = np.sign(np.sum(x * xr, axis=0))
    d[d == 0] = 1.0
    return np.linalg.norm(x * d - xr, axis=0)


def test_c2_headline_matches_oracle(rsvd_lib):
    pkg = rsvd_lib
    w = synth.C2
    A = synth.device_lowrank(w.m, w.n, w.sigma(), w.matrix_seed)
    Ahl = pkg.split_bf16(A)
    with pkg.Plan(w.m, w.n, w.k, w.p, w.q, w.omega_seed, pkg.RSVD_BF16_TC, dtype=pkg.RSVD_BF16X2,
                  residual_passes=1) as pl:
        U, S, V = pl.svd(Ahl)
        U, S, V = pl.svd(Ahl, U, S, V)       # the replayed graph gives the same result
    u, s, v = _np(U), _np(S), _np(V)
    a64 = _np(A)
    del A
    hl = _np(Ahl)
    del Ahl
    torch.cuda.empty_cache()
    hl = hl[: w.m] + hl[w.m:]                   # the stored matrix, hi + lo
    om = philox.gaussian(w.omega_seed, philox.STREAM_OMEGA, w.n, w.l)

    # (1) the precision pattern in float64 (untruncated: sigma_{k+1} for the last gap)
    um, sm, vm, _ = mixed.rsvd(hl, w.l, 0, w.q, om)
    del hl
    sr = sm[: w.k]
    assert np.max(np.abs(s - sr)) <= EPS * sr[0], np.max(np.abs(s - sr)) / sr[0]
    bound = metrics.gap_bound(sr, EPS, c=1.0, s_next=sm[w.k]) + EPS
    du, dv = _vec_dist(u, um[:, : w.k]), _vec_dist(v, vm[:, : w.k])
    assert np.all(du <= bound), (du / bound).max()
    assert np.all(dv <= bound), (dv / bound).max()

    # (2) the method without roundings, on the float32 A
    up, sp, vp, _ = rsvd64.rsvd(a64, w.k, w.p, w.q, om)
    by_design = np.abs(sr - sp)
    assert np.all(np.abs(s - sp) <= by_design + EPS * sp[0])
    e_plain = metrics.fro_error_onepass(a64, up, sp, vp)
    e_gpu = metrics.fro_error_onepass(a64, u, s, v)
    assert (e_gpu - e_plain) / e_plain <= 1e-4, (e_gpu - e_plain) / e_plain
