"""Failure detection without a GPU fault.

* A bounded device wait that runs out: rsvd_wait_selftest waits for a device word that
  nothing sets, with a short limit; the kernel records the timeout and returns, rsvd_sync
  reports RSVD_ERR_TIMEOUT once, and the plan (and the context) keep working.
* Allocation failure: rsvd_debug_fail_alloc makes the n-th device allocation fail on the
  host, as a failed cudaMalloc would; plan creation returns RSVD_ERR_ALLOC for every n
  that lands inside it, and a later creation succeeds.  The backward's workspace (taken by
  its first call) fails the same way and leaves the plan usable.
* Numerical safeguards: a rank-1 input makes the sample matrix rank 1, so every
  Cholesky-QR round floors its trailing pivots; the status bit for it is raised
  (informational, not an error) and the result is finite and exact.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import philox, rsvd64

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_reports(rsvd_lib):
    pkg = rsvd_lib
    m, n, k, p, q = 400, 300, 8, 4, 1
    a, *_ = synth.lowrank(m, n, synth.spectrum_exp(n, 5.0), 3)
    A = torch.tensor(a.astype(np.float32), device="cuda")
    with pkg.Plan(m, n, k, p, q, 9) as pl:
        pkg.rsvd_wait_selftest(pl.handle, 2000)
        assert pkg.rsvd_sync(pl.handle) == pkg.RSVD_ERR_TIMEOUT
        assert pkg.rsvd_sync(pl.handle) == pkg.RSVD_OK           # reported once, then cleared
        U, S, V = pl.svd(A)                                      # the plan still works
    om = philox.gaussian(9, 0, n, k + p)
    _, s_ref, _, _ = rsvd64.rsvd(a.astype(np.float32).astype(np.float64), k, p, q, om)
    assert np.max(np.abs(S.cpu().numpy() - s_ref)) <= 1e-5 * s_ref[0]


@pytest.mark.parametrize("after", [0, 3, 9])
def test_allocation_failure_is_reported(rsvd_lib, after):
    pkg = rsvd_lib
    m, n, k, p, q = 256, 200, 8, 8, 1
    pkg.rsvd_debug_fail_alloc(after)
    try:
        with pytest.raises(pkg.RsvdError) as e:
            pkg.Plan(m, n, k, p, q, 1)
        assert e.value.status == pkg.RSVD_ERR_ALLOC
    finally:
        pkg.rsvd_debug_fail_alloc(-1)
    with pkg.Plan(m, n, k, p, q, 1) as pl:                       # a fresh plan is fine
        A = torch.randn(m, n, device="cuda")
        pl.svd(A)
        pkg.rsvd_debug_fail_alloc(0)                             # the backward's workspace
        try:
            with pytest.raises(pkg.RsvdError) as e:
                pl.backward(A, add_recon=1)
            assert e.value.status == pkg.RSVD_ERR_ALLOC
        finally:
            pkg.rsvd_debug_fail_alloc(-1)
        g = pl.backward(A, add_recon=1)                          # and then it works
        assert torch.isfinite(g).all()


def test_rank_one_sample_floors_the_pivots(rsvd_lib):
    pkg = rsvd_lib
    m, n, k, p, q = 600, 450, 4, 4, 1
    rng = np.random.default_rng(5)
    u = rng.standard_normal(m)
    v = rng.standard_normal(n)
    a = (np.outer(u / np.linalg.norm(u), v / np.linalg.norm(v)) * 3.0).astype(np.float32)
    with pkg.Plan(m, n, k, p, q, 2) as pl:
        U, S, V = pl.svd(torch.tensor(a, device="cuda"), sync=False)
        bits, _ = pkg.rsvd_diagnostics(pl.handle)   # before rsvd_sync clears the word
        assert pkg.rsvd_sync(pl.handle) == pkg.RSVD_OK   # informational, not an error
    s = S.cpu().numpy()
    assert bits & 4                                             # a pivot was floored
    assert np.all(np.isfinite(U.cpu().numpy())) and np.all(np.isfinite(V.cpu().numpy()))
    assert abs(s[0] - 3.0) <= 1e-5 * 3.0 and np.all(np.abs(s[1:]) <= 1e-5 * 3.0)
