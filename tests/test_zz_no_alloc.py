"""The allocation-free tensor-core pass against the plan-based pass.

rsvd_sketch_bf16_noalloc serves callers that cannot allocate device memory
(services that pre-size all device memory at start-up, code running under
stream capture, latency-critical loops that cannot afford cudaMalloc's
implicit synchronisation).  It runs the same kernel as rsvd_sketch on a
bfloat16 plan, with its scratch in a static device array instead of plan
workspace, so on the same inputs the two must agree within the tensor-core
pass tolerance |Y - Y_ref| <= 1e-5 (|A| |X|)_ij -- here on two calls in a row,
since every call reuses (and must re-clear) the same static scratch.

This file is collected last so that a run stopping at the first failure has
already run every other test; it must also pass when run alone.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _ld8(k):
    return (k + 7) // 8 * 8


@pytest.mark.parametrize("m,n,l,transpose", [(1000, 520, 112, 0), (1000, 520, 112, 1),
                                             (4096, 2048, 64, 0), (517, 1000, 32, 1)])
def test_noalloc_pass_matches_plan_pass(rsvd_lib, m, n, l, transpose):
    gen = torch.Generator(device="cuda")
    gen.manual_seed(m + n + l + transpose)
    A = torch.randn(m, n, generator=gen, device="cuda").to(torch.bfloat16)
    K = m if transpose else n
    M = n if transpose else m
    X = torch.randn(K, l, generator=gen, device="cuda")
    # reference: the plan-based pass (rounds X to bfloat16 inside the library)
    Y_ref = torch.empty(M, l, device="cuda")
    with rsvd_lib.Plan(m, n, l, 0, 0, 1, rsvd_lib.RSVD_BF16_TC) as pl:
        rsvd_lib.rsvd_sketch(pl.handle, A, transpose, X, Y_ref)
        assert rsvd_lib.rsvd_sync(pl.handle) == rsvd_lib.RSVD_OK
    # the same operand, transposed to bfloat16 by the caller
    ldxt = _ld8(K)
    Xt = torch.zeros(l, ldxt, device="cuda", dtype=torch.bfloat16)
    Xt[:, :K] = X.t().to(torch.bfloat16)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    a64 = A.double()
    op = a64.t() if transpose else a64
    bound = 1e-5 * (op.abs() @ Xt[:, :K].double().t().abs())
    for _ in range(2):
        Y = torch.full((M, l), float("nan"), device="cuda")
        rsvd_lib.rsvd_sketch_bf16_noalloc(A, m, n, n, transpose, Xt, ldxt, l, Y, status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.all((Y.double() - Y_ref.double()).abs() <= bound)


def test_noalloc_rejects_sizes_beyond_its_scratch(rsvd_lib):
    A = torch.zeros(256, 256, device="cuda", dtype=torch.bfloat16)
    Xt = torch.zeros(144, 256, device="cuda", dtype=torch.bfloat16)
    Y = torch.zeros(256, 144, device="cuda")
    with pytest.raises(rsvd_lib.RsvdError) as e:
        rsvd_lib.rsvd_sketch_bf16_noalloc(A, 256, 256, 256, 0, Xt, 256, 144, Y)
    assert e.value.status == rsvd_lib.RSVD_ERR_INVALID_ARG
    with pytest.raises(rsvd_lib.RsvdError) as e:      # l not a multiple of 16
        rsvd_lib.rsvd_sketch_bf16_noalloc(A, 256, 256, 256, 0, Xt, 256, 40, Y)
    assert e.value.status == rsvd_lib.RSVD_ERR_INVALID_ARG
