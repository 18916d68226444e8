"""The C3 and C4 workloads at their full sizes, as the bench times them, against the float64
oracle (oracle.mixed: Algorithm 4.4 + 5.1 with the roundings the tensor-core form makes by
design, run on the stored bfloat16 A with the same test matrix).

  * C4: 32768 x 32768, sigma_j = j^-0.5, k = 236, p = 20, q = 1; Gaussian and SRFT test
    matrices (the SRFT's Omega is the oracle's explicit real SRFT of the same draws).
  * C3: 262144 x 4096, sigma_j = max(e^-(j-1)/20, 1e-6) + N(0, 1e-8) noise, k = 64, p = 16,
    the q = 2 multi-pass form, and the single pass against oracle.single_pass.

What remains between the GPU and the oracle is float32 arithmetic, held to the library's
float32 targets: |sigma_j - sigma_j^ref| <= 1e-5 sigma_1, and after sign alignment
||x_j - x_j^ref|| <= 1e-5 sigma_1 / gap_j + 1e-5 (Wedin), gap_j from the oracle's values
(sigma_{k+1} for the last).  Each case holds the 2-8.6 GB float64 copy of A on the host.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import metrics, mixed, philox, srft

pytestmark = pytest.mark.gpu

EPS = 1e-5


def _np(t):
    return t.detach().double().cpu().numpy()


def _vec_dist(x, xr):
    d = np.sign(np.sum(x * xr, axis=0))
    d[d == 0] = 1.0
    return np.linalg.norm(x * d - xr, axis=0)


def _check(u, s, v, um, sm, vm, k):
    sr = sm[:k]
    err = np.max(np.abs(s - sr)) / sr[0]
    print(f"max |dsigma| / sigma_1 = {err:.2e}")
    assert err <= EPS
    bound = metrics.gap_bound(sr, EPS, c=1.0, s_next=sm[k]) + EPS
    du, dv = _vec_dist(u, um[:, :k]), _vec_dist(v, vm[:, :k])
    assert np.all(du <= bound), (du / bound).max()
    assert np.all(dv <= bound), (dv / bound).max()


def _run(pkg, w, A, q, **plan_kw):
    with pkg.Plan(w.m, w.n, w.k, w.p, q, w.omega_seed, pkg.RSVD_BF16_TC, **plan_kw) as pl:
        U, S, V = pl.svd(A)
        assert pkg.rsvd_sync(pl.handle) == pkg.RSVD_OK
    return _np(U), _np(S), _np(V)


@pytest.mark.parametrize("test_matrix", ["gaussian", "srft"])
def test_c4_full_size(rsvd_lib, test_matrix):
    pkg = rsvd_lib
    w = synth.C4
    A = synth.device_lowrank(w.m, w.n, w.sigma(), w.matrix_seed).to(torch.bfloat16)
    kw = {"test_matrix": pkg.RSVD_SRFT} if test_matrix == "srft" else {}
    u, s, v = _run(pkg, w, A, w.q, **kw)
    a64 = _np(A)
    del A
    torch.cuda.empty_cache()
    if test_matrix == "srft":
        signs, freqs = srft.draw(w.omega_seed, w.n, w.l // 2)
        om = srft.omega_real(signs, freqs)
    else:
        om = philox.gaussian(w.omega_seed, philox.STREAM_OMEGA, w.n, w.l)
    um, sm, vm, _ = mixed.rsvd(a64, w.l, 0, w.q, om)
    del a64
    _check(u, s, v, um, sm, vm, w.k)


def test_c3_multi_pass_full_size(rsvd_lib):
    pkg = rsvd_lib
    w = synth.C3
    q = 2
    A = synth.device_lowrank(w.m, w.n, w.sigma(), w.matrix_seed, noise_std=w.noise_std()).to(torch.bfloat16)
    u, s, v = _run(pkg, w, A, q)
    a64 = _np(A)
    del A
    torch.cuda.empty_cache()
    om = philox.gaussian(w.omega_seed, philox.STREAM_OMEGA, w.n, w.l)
    um, sm, vm, _ = mixed.rsvd(a64, w.l, 0, q, om)
    del a64
    _check(u, s, v, um, sm, vm, w.k)


def test_c3_single_pass_full_size(rsvd_lib):
    """The single pass (Section 5.5) at the full C3 size against oracle.single_pass on the
    library's own Omega and Psi (read back through the C ABI, bfloat16 as the passes use
    them): singular values within 2 u32 (kappa(X1)^2 + kappa(X2)^2) sigma_1 (the first-order
    bound of tests/test_gpu_single_pass.py), and the relative reconstruction error within
    2 % of the oracle's."""
    import os
    import sys

    sys.path.insert(0, os.path.dirname(__file__))
    from test_gpu_single_pass import U32, _oracle, psi_cols

    pkg = rsvd_lib
    w = synth.C3
    A = synth.device_lowrank(w.m, w.n, w.sigma(), w.matrix_seed, noise_std=w.noise_std()).to(torch.bfloat16)
    with pkg.Plan(w.m, w.n, w.k, w.p, 0, w.omega_seed, pkg.RSVD_BF16_TC, single_pass=1) as pl:
        U, S, V = pl.svd(A)
        om = torch.zeros(w.n, w.l, device="cuda")
        pkg.rsvd_get_omega(pl.handle, om)
        assert pkg.rsvd_sync(pl.handle) == pkg.RSVD_OK
    lt = psi_cols(w.m, w.n, w.l)
    psi = torch.zeros(w.m, lt, device="cuda")
    pkg.rsvd_draw_gaussian(w.omega_seed, 1, w.m, lt, psi, lt)
    torch.cuda.synchronize()
    u, s, v = _np(U), _np(S), _np(V)
    om64 = _np(om.to(torch.bfloat16))
    psi64 = _np(psi.to(torch.bfloat16))
    a64 = _np(A)
    del A, psi
    torch.cuda.empty_cache()
    ur, sr, vr, sb, kap = _oracle(a64, w.k, om64, psi64)
    tol = 2 * U32 * kap * sr[0]
    err = np.max(np.abs(s - sr))
    e_gpu = metrics.fro_error_onepass(a64, u, s, v)
    e_ref = metrics.fro_error_onepass(a64, ur, sr, vr)
    na = float(np.sqrt(np.sum(a64 * a64)))
    print(f"C3 single pass: max dsigma / sigma_1 {err / sr[0]:.2e} (tol {tol / sr[0]:.2e}), "
          f"relative error {e_gpu / na:.4f} (oracle {e_ref / na:.4f})")
    assert err <= tol
    assert abs(e_gpu - e_ref) <= 0.02 * e_ref
