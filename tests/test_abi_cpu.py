"""C ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every entry point include/rsvd.h declares, and rejects bad arguments on the
host before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    import paper_0909_4061_gb300 as p
    from paper_0909_4061_gb300 import build

    build.build()
    p.lib()
    return p


def _declared():
    with open(os.path.join(ROOT, "include", "rsvd.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"RSVD_API\s+[\w\s\*]+?\b(rsvd_\w+)\s*\(", text)))


def test_header_declares_what_binding_expects(pkg):
    assert _declared() == sorted(pkg.EXPORTS)


def test_every_declared_symbol_is_exported(pkg):
    handle = ctypes.CDLL(pkg.LIB_PATH)
    for name in _declared():
        assert hasattr(handle, name), name


def test_only_the_c_abi_is_exported(pkg):
    import subprocess

    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB_PATH], capture_output=True,
                         text=True).stdout
    funcs = [line.split()[-1] for line in out.splitlines() if " T " in line]
    assert funcs and all(f.startswith("rsvd_") for f in funcs), funcs


def test_options_default_and_status_strings(pkg):
    o = pkg.rsvd_options_default()
    assert (o.dtype_A, o.precision, o.test_matrix, o.orth_rounds, o.lda) == (0, 0, 0, 3, 0)
    assert pkg.status_string(0) == "success"
    assert "invalid" in pkg.status_string(1)
    assert pkg.status_string(99) == "unknown status"


@pytest.mark.parametrize("m,n,k,p,q", [(0, 10, 1, 0, 0), (10, 10, 0, 1, 0), (10, 10, 5, 6, 0),
                                       (10, 10, 3, -1, 0), (10, 10, 3, 1, -1), (400, 400, 250, 10, 0)])
def test_plan_create_rejects_bad_sizes_on_host(pkg, m, n, k, p, q):
    with pytest.raises(pkg.RsvdError) as e:
        pkg.rsvd_plan_create(m, n, k, p, q, 0, None, 0)
    assert e.value.status == pkg.RSVD_ERR_INVALID_ARG


def test_plan_create_rejects_bad_options_on_host(pkg):
    o = pkg.rsvd_options_default()
    o.orth_rounds = 5
    with pytest.raises(pkg.RsvdError) as e:
        pkg.rsvd_plan_create(100, 80, 5, 5, 1, 0, o, 0)
    assert e.value.status == pkg.RSVD_ERR_INVALID_ARG
    o = pkg.rsvd_options_default()
    o.lda = 10      # lda < n
    with pytest.raises(pkg.RsvdError) as e:
        pkg.rsvd_plan_create(100, 80, 5, 5, 1, 0, o, 0)
    assert e.value.status == pkg.RSVD_ERR_INVALID_ARG
    o = pkg.rsvd_options_default()
    o.precision = pkg.RSVD_BF16_TC   # bf16 tensor-core path needs a bf16 A
    with pytest.raises(pkg.RsvdError) as e:
        pkg.rsvd_plan_create(100, 80, 5, 5, 1, 0, o, 0)
    assert e.value.status == pkg.RSVD_ERR_INVALID_ARG
    # SRFT: l real columns are l / 2 frequencies of an even-length DFT
    for m, n, k, p in [(100, 80, 5, 4), (100, 81, 5, 5), (100, 8, 6, 2)]:
        o = pkg.rsvd_options_default()
        o.test_matrix = pkg.RSVD_SRFT
        with pytest.raises(pkg.RsvdError) as e:
            pkg.rsvd_plan_create(m, n, k, p, 1, 0, o, 0)
        assert e.value.status == pkg.RSVD_ERR_INVALID_ARG, (m, n, k, p)
    o = pkg.rsvd_options_default()
    o.small_svd = 3
    with pytest.raises(pkg.RsvdError) as e:
        pkg.rsvd_plan_create(100, 80, 5, 5, 1, 0, o, 0)
    assert e.value.status == pkg.RSVD_ERR_INVALID_ARG
    # the residual of A in every pass needs A stored as hi + lo
    assert pkg.rsvd_options_default().residual_passes == 0
    for dtype, rp in [(pkg.RSVD_BF16, 1), (pkg.RSVD_BF16, 2), (pkg.RSVD_BF16X2, 3), (pkg.RSVD_F32, 1)]:
        o = pkg.rsvd_options_default()
        o.precision = pkg.RSVD_PLAIN_FP32 if dtype == pkg.RSVD_F32 else pkg.RSVD_BF16_TC
        o.dtype_A = dtype
        o.residual_passes = rp
        with pytest.raises(pkg.RsvdError) as e:
            pkg.rsvd_plan_create(100, 80, 5, 5, 1, 0, o, 0)
        assert e.value.status == pkg.RSVD_ERR_INVALID_ARG, (dtype, rp)


def test_null_pointer_arguments(pkg):
    lib = pkg.lib()
    assert lib.rsvd_plan_create(None, 10, 10, 1, 0, 0, 0, None, None) == pkg.RSVD_ERR_INVALID_ARG
    assert lib.rsvd_svd(None, None, None, None, None) == pkg.RSVD_ERR_INVALID_ARG
    assert lib.rsvd_plan_destroy(None) == pkg.RSVD_OK
    assert lib.rsvd_draw_gaussian(0, 0, 10, 10, None, 10, None) == pkg.RSVD_ERR_INVALID_ARG


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_0909_4061_gb300 as p

    monkeypatch.setattr(p, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(p, "_lib", None)
    with pytest.raises(p.RsvdUnavailable):
        p.lib()
