"""GPU parity of the adaptive range finder (blocked Algorithm 4.2) against oracle.adaptive.

Both sides take the same sample stream (the Gaussian columns of Philox stream 3 for the
plan's seed, n x (l_p + block), read from the oracle's generator), so they make the same
stopping decisions as long as no block's estimate sits at the threshold (each tolerance
below is placed a factor of 3 or more away from every estimate the oracle sees).  Compared:
  * the rank (an integer decision: exact),
  * the first block as a subspace: ||(I - Q_ref Q_ref^T) Q_1|| <= 1e-4.  Later blocks
    come from projected samples (I - Q Q^T) A w whose size is that of the singular values
    left, far below ||A|| ||w||: float32 cancellation leaves them a relative error of
    about 2^-24 ||A|| ||w|| / ||(I - Q Q^T) A w|| (1e-3 and more here), so they are held
    to what they must achieve instead,
  * the posterior estimate of the last block (relative 1e-3 + 1e-6 of ||A||): it depends
    on the whole basis, and a direction missing from it shows as a larger estimate,
  * the error ||(I - Q Q^T) A||_2 against the oracle's (relative 5 % + 1e-5 ||A||) and
    the guarantee itself, ||(I - Q Q^T) A||_2 <= eps.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import adaptive, metrics, philox

pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().double().cpu().numpy()


def _omega(seed, n, lp, block, bf16):
    om = philox.gaussian(seed, 3, n, lp + block)
    if bf16:
        om = torch.tensor(om, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    return om


def _estimates(a, om, block, cap):
    """The oracle's estimate max_i ||Y[:, i]|| for every block up to the cap (eps = 0)."""
    q = np.zeros((a.shape[0], 0))
    y = a @ om[:, :block]
    out, t = [], 1
    while True:
        out.append(float(np.max(np.linalg.norm(y, axis=0))))
        if q.shape[1] + block > cap:
            return out
        q = np.hstack([q, adaptive.orth_block(q, y)])
        y = adaptive.project_out(q, a @ om[:, t * block:(t + 1) * block])
        t += 1


# (m, n, block, decay of the spectrum exp(-i / decay), the block j at which to stop, bf16)
# The tolerance is set between the oracle's estimates of blocks j - 1 and j, at their
# geometric mean, so that every decision sits at least a factor 3 from the threshold.
@pytest.mark.parametrize("m,n,block,decay,j,prec", [(1500, 900, 16, 4.0, 3, 0), (1500, 900, 16, 4.0, 2, 0),
                                                    (1100, 1300, 32, 8.0, 3, 0), (2000, 1024, 16, 4.0, 2, 1)])
def test_adaptive_matches_oracle(rsvd_lib, m, n, block, decay, j, prec):
    pkg = rsvd_lib
    sig = np.exp(-np.arange(min(m, n)) / decay)
    a, *_ = synth.lowrank(m, n, sig, m + n)
    k, p, seed = 112, 16, 23
    cap = k + p
    bf16 = prec == pkg.RSVD_BF16_TC
    a32 = a.astype(np.float32)
    if bf16:
        a32 = torch.tensor(a32).to(torch.bfloat16).float().numpy()
    a64 = a32.astype(np.float64)
    om = _omega(seed, n, cap, block, bf16)
    e = _estimates(a64, om, block, cap)
    assert min(e[:j]) >= 9 * e[j]
    eps = float(np.sqrt(min(e[:j]) * e[j])) * adaptive.THRESHOLD_FACTOR
    q_ref, est_ref = adaptive.adaptive_range_finder(a64, eps, om, block, cap)
    assert q_ref.shape[1] == j * block
    with pkg.Plan(m, n, k, p, 0, seed, prec) as pl:
        A = torch.tensor(a32, device="cuda", dtype=torch.bfloat16 if bf16 else torch.float32)
        Q = torch.zeros(m, cap, device="cuda")
        rank, est = pkg.rsvd_range_finder_adaptive(pl.handle, A, eps, block, Q, cap)
        assert pkg.rsvd_sync(pl.handle) == pkg.RSVD_OK
    q = _np(Q)[:, :rank]
    print(f"adaptive {m}x{n} eps={eps:.2e} block={block} prec={prec}: rank {rank} (oracle {q_ref.shape[1]}), "
          f"estimate {est:.3e} (oracle {est_ref:.3e})")
    assert rank == q_ref.shape[1]
    q1, r1 = q[:, :block], q_ref[:, :block]
    assert np.linalg.norm(q1 - r1 @ (r1.T @ q1), 2) <= 1e-4
    assert abs(est - est_ref) <= 1e-3 * est_ref + 1e-6 * sig[0]
    err, err_ref = metrics.projection_error(a64, q), metrics.projection_error(a64, q_ref)
    assert abs(err - err_ref) <= 0.05 * err_ref + 1e-5 * sig[0]
    assert err <= eps
    assert metrics.orthonormality(q) <= 2e-5


def test_adaptive_exact_rank(rsvd_lib):
    pkg = rsvd_lib
    m, n, r, block = 800, 600, 20, 16
    a, *_ = synth.lowrank(m, n, np.linspace(2.0, 0.5, r), 5)
    with pkg.Plan(m, n, 80, 16, 0, 4) as pl:
        Q = torch.zeros(m, 96, device="cuda")
        rank, est = pkg.rsvd_range_finder_adaptive(pl.handle, torch.tensor(a.astype(np.float32), device="cuda"),
                                                   1e-4, block, Q, 96)
        pkg.rsvd_sync(pl.handle)
    q = _np(Q)[:, :rank]
    assert rank == 32
    assert metrics.projection_error(a, q) <= 1e-5 * np.linalg.norm(a, 2)
