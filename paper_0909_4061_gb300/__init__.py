"""Python binding of the GB300 randomized range finder / randomized SVD library.

Argument marshalling only: every function below forwards to the C ABI of
include/rsvd.h (libpaper_rsvd.so, built in-tree by ``paper_0909_4061_gb300.build``)
and every step of the computation runs in the library's CUDA kernels.  The
functions carry the C names; ``Plan`` and ``svd`` are thin conveniences that
take torch CUDA tensors (device memory and the current stream come from torch).

There is no CPU fallback: if the shared library is missing or cannot be
loaded, every call raises ``RsvdUnavailable``.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpaper_rsvd.so")

RSVD_OK = 0
RSVD_ERR_INVALID_ARG = 1
RSVD_ERR_ALLOC = 2
RSVD_ERR_CUDA = 3
RSVD_ERR_NUMERICAL = 4
RSVD_ERR_NONFINITE = 5
RSVD_ERR_TIMEOUT = 6
RSVD_ERR_UNSUPPORTED = 7

RSVD_F32, RSVD_BF16, RSVD_BF16X2 = 0, 1, 2
RSVD_GAUSSIAN, RSVD_SRFT, RSVD_GSRFT = 0, 1, 2
RSVD_PLAIN_FP32, RSVD_BF16_TC = 0, 1
RSVD_SMALL_AUTO, RSVD_SMALL_ONE_CTA, RSVD_SMALL_CLUSTER = 0, 1, 2
RSVD_EIG_DIRECT, RSVD_EIG_NYSTROM = 0, 1

# every symbol include/rsvd.h declares (checked by the CPU tests)
EXPORTS = (
    "rsvd_options_default", "rsvd_plan_create", "rsvd_plan_destroy", "rsvd_workspace_bytes",
    "rsvd_range_finder", "rsvd_svd", "rsvd_svd_host", "rsvd_svd_backward", "rsvd_get_omega",
    "rsvd_set_omega", "rsvd_sync", "rsvd_status_string", "rsvd_draw_gaussian", "rsvd_sketch",
    "rsvd_orthonormalize", "rsvd_small_svd", "rsvd_profile", "rsvd_profile_read",
    "rsvd_diagnostics", "rsvd_sketch_bf16_noalloc", "rsvd_convert_a",
    "rsvd_batched_plan_create", "rsvd_batched_plan_destroy", "rsvd_batched_svd", "rsvd_batched_sync",
    "rsvd_batched_svd_backward", "rsvd_wait_selftest", "rsvd_debug_fail_alloc",
    "rsvd_batched_tuning", "rsvd_sketch_srft", "rsvd_range_finder_adaptive", "rsvd_eig",
    "rsvd_row_id", "rsvd_svd_row_extraction",
)

RSVD_STEP_DRAW, RSVD_STEP_PASS, RSVD_STEP_ORTH = 0, 1, 2
RSVD_STEP_SMALL_SVD, RSVD_STEP_LIFT, RSVD_STEP_CONVERT, RSVD_STEP_ID, RSVD_NUM_STEPS = 3, 4, 5, 6, 7
STEP_NAMES = ("draw", "pass", "orth", "small_svd", "lift", "convert", "id")


class RsvdUnavailable(ImportError):
    pass


class RsvdError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


class Options(ctypes.Structure):
    _fields_ = [
        ("dtype_A", ctypes.c_int32),
        ("test_matrix", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("single_pass", ctypes.c_int32),
        ("recompute", ctypes.c_int32),
        ("orth_rounds", ctypes.c_int32),
        ("lda", ctypes.c_int64),
        ("small_svd", ctypes.c_int32),
        ("residual_passes", ctypes.c_int32),
        ("psi_cols", ctypes.c_int32),
        ("srft_fft", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("host_f32", ctypes.c_int32),
    ]


_lib = None

_c = ctypes
_P = ctypes.c_void_p
_SIGS = {
    "rsvd_options_default": (None, [_P]),
    "rsvd_plan_create": (_c.c_int, [_P, _c.c_int64, _c.c_int64, _c.c_int32, _c.c_int32, _c.c_int32,
                                    _c.c_uint64, _P, _P]),
    "rsvd_plan_destroy": (_c.c_int, [_P]),
    "rsvd_workspace_bytes": (_c.c_int, [_P, _P]),
    "rsvd_range_finder": (_c.c_int, [_P, _P, _P, _c.c_int64]),
    "rsvd_svd": (_c.c_int, [_P, _P, _P, _P, _P]),
    "rsvd_svd_host": (_c.c_int, [_P, _P, _P, _P, _P]),
    "rsvd_svd_backward": (_c.c_int, [_P, _P, _P, _P, _P, _c.c_int32, _P]),
    "rsvd_get_omega": (_c.c_int, [_P, _P]),
    "rsvd_set_omega": (_c.c_int, [_P, _P]),
    "rsvd_sync": (_c.c_int, [_P]),
    "rsvd_status_string": (_c.c_char_p, [_c.c_int]),
    "rsvd_draw_gaussian": (_c.c_int, [_c.c_uint64, _c.c_uint32, _c.c_int64, _c.c_int64, _P,
                                      _c.c_int64, _P]),
    "rsvd_sketch": (_c.c_int, [_P, _P, _c.c_int32, _P, _P]),
    "rsvd_orthonormalize": (_c.c_int, [_P, _c.c_int64, _P, _P]),
    "rsvd_small_svd": (_c.c_int, [_P, _P, _P, _P, _P]),
    "rsvd_profile": (_c.c_int, [_P, _c.c_uint32]),
    "rsvd_profile_read": (_c.c_int, [_P, _P, _P, _c.c_int32]),
    "rsvd_diagnostics": (_c.c_int, [_P, _P, _c.c_int32]),
    "rsvd_convert_a": (_c.c_int, [_P, _c.c_int64, _c.c_int64, _c.c_int64, _P, _c.c_int64,
                                  _c.c_int32, _P]),
    "rsvd_sketch_bf16_noalloc": (_c.c_int, [_P, _c.c_int64, _c.c_int64, _c.c_int64, _c.c_int32, _P,
                                            _c.c_int64, _c.c_int32, _P, _P, _P]),
    "rsvd_batched_plan_create": (_c.c_int, [_P, _c.c_int32, _P, _P, _P, _c.c_int32, _c.c_int32,
                                            _c.c_int32, _c.c_uint64, _P, _P]),
    "rsvd_batched_plan_destroy": (_c.c_int, [_P]),
    "rsvd_batched_svd": (_c.c_int, [_P, _P, _P, _P, _P]),
    "rsvd_batched_sync": (_c.c_int, [_P, _P]),
    "rsvd_batched_svd_backward": (_c.c_int, [_P, _P, _P]),
    "rsvd_wait_selftest": (_c.c_int, [_P, _c.c_uint32]),
    "rsvd_batched_tuning": (_c.c_int, [_P, _P, _P, _P]),
    "rsvd_sketch_srft": (_c.c_int, [_P, _P, _P]),
    "rsvd_eig": (_c.c_int, [_P, _P, _c.c_int32, _P, _P]),
    "rsvd_row_id": (_c.c_int, [_P, _P, _c.c_int64, _P, _P, _c.c_int64]),
    "rsvd_svd_row_extraction": (_c.c_int, [_P, _P, _P, _P, _P]),
    "rsvd_range_finder_adaptive": (_c.c_int, [_P, _P, _c.c_float, _c.c_int32, _P, _c.c_int64, _P, _P]),
    "rsvd_debug_fail_alloc": (None, [_c.c_int32]),
}


def lib():
    """The loaded shared library (raises RsvdUnavailable when it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RsvdUnavailable(
                f"{LIB_PATH} is missing: build it with `python -m paper_0909_4061_gb300.build` "
                "(or __graft_entry__.build()); there is no CPU fallback")
        try:
            handle = ctypes.CDLL(LIB_PATH)
        except OSError as e:
            raise RsvdUnavailable(f"cannot load {LIB_PATH}: {e}") from e
        for name, (res, args) in _SIGS.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def status_string(status: int) -> str:
    try:
        return lib().rsvd_status_string(int(status)).decode()
    except RsvdUnavailable:
        return f"status {status}"


def _check(status: int, where: str):
    if status != RSVD_OK:
        raise RsvdError(status, where)


def _ptr(x):
    """Device or host address of a torch tensor / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- C ABI, one wrapper per entry point -----------------------------------------


def rsvd_options_default() -> Options:
    o = Options()
    lib().rsvd_options_default(ctypes.byref(o))
    return o


def rsvd_plan_create(m, n, k, p, q, seed, opt: Options | None = None, stream=None):
    h = ctypes.c_void_p()
    st = lib().rsvd_plan_create(ctypes.byref(h), int(m), int(n), int(k), int(p), int(q),
                                int(seed) & 0xFFFFFFFFFFFFFFFF,
                                ctypes.byref(opt) if opt is not None else None, _stream(stream))
    _check(st, "rsvd_plan_create")
    return h


def rsvd_plan_destroy(plan):
    _check(lib().rsvd_plan_destroy(plan), "rsvd_plan_destroy")


def rsvd_workspace_bytes(plan) -> int:
    v = ctypes.c_size_t()
    _check(lib().rsvd_workspace_bytes(plan, ctypes.byref(v)), "rsvd_workspace_bytes")
    return v.value


def rsvd_range_finder(plan, A, Q, ldq):
    _check(lib().rsvd_range_finder(plan, _ptr(A), _ptr(Q), int(ldq)), "rsvd_range_finder")


def rsvd_svd(plan, A, U, S, V):
    _check(lib().rsvd_svd(plan, _ptr(A), _ptr(U), _ptr(S), _ptr(V)), "rsvd_svd")


def rsvd_svd_host(plan, A_host, U_host, S_host, V_host):
    _check(lib().rsvd_svd_host(plan, _ptr(A_host), _ptr(U_host), _ptr(S_host), _ptr(V_host)),
           "rsvd_svd_host")


def rsvd_svd_backward(plan, A, gU, gS, gV, add_recon, gA):
    _check(lib().rsvd_svd_backward(plan, _ptr(A), _ptr(gU), _ptr(gS), _ptr(gV), int(add_recon),
                                   _ptr(gA)), "rsvd_svd_backward")


def rsvd_get_omega(plan, Omega):
    _check(lib().rsvd_get_omega(plan, _ptr(Omega)), "rsvd_get_omega")


def rsvd_set_omega(plan, Omega):
    _check(lib().rsvd_set_omega(plan, _ptr(Omega)), "rsvd_set_omega")


def rsvd_sync(plan) -> int:
    """Returns the status code (does not raise) so callers can test device-side errors."""
    return lib().rsvd_sync(plan)


def rsvd_wait_selftest(plan, spins):
    _check(lib().rsvd_wait_selftest(plan, int(spins)), "rsvd_wait_selftest")


def rsvd_debug_fail_alloc(after):
    lib().rsvd_debug_fail_alloc(int(after))


def rsvd_status_string(status: int) -> str:
    return status_string(status)


def rsvd_draw_gaussian(seed, stream_id, rows, cols, out, ld, stream=None):
    _check(lib().rsvd_draw_gaussian(int(seed) & 0xFFFFFFFFFFFFFFFF, int(stream_id), int(rows),
                                    int(cols), _ptr(out), int(ld), _stream(stream)),
           "rsvd_draw_gaussian")


def rsvd_sketch(plan, A, transpose, X, Y):
    _check(lib().rsvd_sketch(plan, _ptr(A), int(transpose), _ptr(X), _ptr(Y)), "rsvd_sketch")


def rsvd_range_finder_adaptive(plan, A, eps, block, Q, ldq):
    """Returns (rank, estimate); Q's first `rank` columns are the basis."""
    rank = ctypes.c_int32(0)
    est = ctypes.c_float(0.0)
    _check(lib().rsvd_range_finder_adaptive(plan, _ptr(A), float(eps), int(block), _ptr(Q), int(ldq),
                                            ctypes.byref(rank), ctypes.byref(est)),
           "rsvd_range_finder_adaptive")
    return int(rank.value), float(est.value)


def rsvd_row_id(plan, Y, ldy, J, X, ldx):
    _check(lib().rsvd_row_id(plan, _ptr(Y), int(ldy), _ptr(J), _ptr(X), int(ldx)), "rsvd_row_id")


def rsvd_svd_row_extraction(plan, A, U, S, V):
    _check(lib().rsvd_svd_row_extraction(plan, _ptr(A), _ptr(U), _ptr(S), _ptr(V)),
           "rsvd_svd_row_extraction")


def rsvd_eig(plan, A, method, U, Lambda):
    _check(lib().rsvd_eig(plan, _ptr(A), int(method), _ptr(U), _ptr(Lambda)), "rsvd_eig")


def rsvd_sketch_srft(plan, A, Y):
    _check(lib().rsvd_sketch_srft(plan, _ptr(A), _ptr(Y)), "rsvd_sketch_srft")


def rsvd_orthonormalize(plan, rows, Y, R=None):
    _check(lib().rsvd_orthonormalize(plan, int(rows), _ptr(Y), _ptr(R)), "rsvd_orthonormalize")


def rsvd_small_svd(plan, X, Ut, S, W):
    _check(lib().rsvd_small_svd(plan, _ptr(X), _ptr(Ut), _ptr(S), _ptr(W)), "rsvd_small_svd")


def rsvd_profile(plan, mask):
    _check(lib().rsvd_profile(plan, int(mask)), "rsvd_profile")


def rsvd_profile_read(plan):
    """Returns ({step name: ms}, {step name: kernel launches})."""
    ms = (ctypes.c_float * RSVD_NUM_STEPS)()
    cnt = (ctypes.c_int64 * RSVD_NUM_STEPS)()
    _check(lib().rsvd_profile_read(plan, ms, cnt, RSVD_NUM_STEPS), "rsvd_profile_read")
    return ({STEP_NAMES[i]: ms[i] for i in range(RSVD_NUM_STEPS)},
            {STEP_NAMES[i]: cnt[i] for i in range(RSVD_NUM_STEPS)})


def rsvd_diagnostics(plan):
    """Returns (status bits seen, largest Jacobi sweep count) since the last call."""
    out = (ctypes.c_uint32 * 2)()
    _check(lib().rsvd_diagnostics(plan, out, 2), "rsvd_diagnostics")
    return int(out[0]), int(out[1])


def rsvd_convert_a(A, m, n, lda, out, ldo, with_lo, stream=None):
    _check(lib().rsvd_convert_a(_ptr(A), int(m), int(n), int(lda), _ptr(out), int(ldo),
                                int(with_lo), _stream(stream)), "rsvd_convert_a")


def rsvd_sketch_bf16_noalloc(A, m, n, lda, transpose, Xt, ldxt, l, Y, status=None, stream=None):
    """One tensor-core pass that allocates nothing (see include/rsvd.h)."""
    _check(lib().rsvd_sketch_bf16_noalloc(_ptr(A), int(m), int(n), int(lda), int(transpose),
                                          _ptr(Xt), int(ldxt), int(l), _ptr(Y), _ptr(status),
                                          _stream(stream)), "rsvd_sketch_bf16_noalloc")


# ---- torch conveniences -------------------------------------------------------------


class Plan:
    """Owns one rsvd plan; tensors are torch CUDA tensors (row-major, contiguous)."""

    def __init__(self, m, n, k, p=10, q=1, seed=0, precision=RSVD_PLAIN_FP32, orth_rounds=3,
                 lda=0, stream=None, test_matrix=RSVD_GAUSSIAN, single_pass=0, dtype=None,
                 small_svd=RSVD_SMALL_AUTO, residual_passes=0, host_f32=0, recompute=0, psi_cols=0,
                 srft_fft=0):
        o = rsvd_options_default()
        o.srft_fft = srft_fft
        o.psi_cols = psi_cols
        o.host_f32 = host_f32
        o.recompute = recompute
        o.small_svd = small_svd
        o.residual_passes = residual_passes
        o.precision = precision
        if dtype is None:
            dtype = RSVD_BF16 if precision == RSVD_BF16_TC else RSVD_F32
        o.dtype_A = dtype
        o.orth_rounds = orth_rounds
        o.lda = lda
        o.test_matrix = test_matrix
        o.single_pass = single_pass
        self.m, self.n, self.k, self.p, self.q = int(m), int(n), int(k), int(p), int(q)
        self.l = self.k + self.p
        self.options = o
        self.handle = rsvd_plan_create(m, n, k, p, q, seed, o, stream)

    def close(self):
        if self.handle is not None:
            rsvd_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def svd(self, A, U=None, S=None, V=None, sync=True):
        import torch

        dev = A.device
        U = U if U is not None else torch.empty(self.m, self.k, device=dev, dtype=torch.float32)
        S = S if S is not None else torch.empty(self.k, device=dev, dtype=torch.float32)
        V = V if V is not None else torch.empty(self.n, self.k, device=dev, dtype=torch.float32)
        rsvd_svd(self.handle, A, U, S, V)
        if sync:
            _check(rsvd_sync(self.handle), "rsvd_svd (device)")
        return U, S, V

    def range_finder(self, A, Q=None, sync=True):
        import torch

        Q = Q if Q is not None else torch.empty(self.m, self.l, device=A.device, dtype=torch.float32)
        rsvd_range_finder(self.handle, A, Q, Q.stride(0))
        if sync:
            _check(rsvd_sync(self.handle), "rsvd_range_finder (device)")
        return Q

    def sync(self):
        _check(rsvd_sync(self.handle), "rsvd_sync")

    def backward(self, A, gU=None, gS=None, gV=None, add_recon=0, gA=None, sync=True):
        """gA (m x n float32) for the cotangents of the last svd() on A (see rsvd.h)."""
        import torch

        gA = gA if gA is not None else torch.empty(self.m, self.n, device=A.device, dtype=torch.float32)
        rsvd_svd_backward(self.handle, A, gU, gS, gV, add_recon, gA)
        if sync:
            _check(rsvd_sync(self.handle), "rsvd_svd_backward (device)")
        return gA

    def stored(self, A):
        """A (float32 CUDA tensor) in the plan's storage: itself for float32 plans, else the
        library's bfloat16 (or hi + lo) conversion."""
        import torch

        dt = self.options.dtype_A
        if dt == RSVD_F32:
            return A
        if dt == RSVD_BF16X2:
            return split_bf16(A)
        out = torch.empty(self.m, self.n, device=A.device, dtype=torch.bfloat16)
        rsvd_convert_a(A, self.m, self.n, A.stride(0), out, self.n, 0)
        return out


def _autograd_function():
    import torch

    class RSVDFunction(torch.autograd.Function):
        """(U, S, V) = rsvd_svd(A) with rsvd_svd_backward as the adjoint (test matrix fixed).

        A is a float32 CUDA tensor; the plan stores it as its dtype requires (the library's
        conversion).  The backward hands the cotangents of U, S and V (None where an output
        is unused) to rsvd_svd_backward; no arithmetic happens here."""

        @staticmethod
        def forward(ctx, A, plan):
            As = plan.stored(A.detach().contiguous())
            U, S, V = plan.svd(As)
            ctx.plan, ctx.stored = plan, As
            ctx.set_materialize_grads(False)
            return U, S, V

        @staticmethod
        def backward(ctx, gU, gS, gV):
            c = (lambda t: None if t is None else t.contiguous())
            gA = ctx.plan.backward(ctx.stored, c(gU), c(gS), c(gV))
            return gA, None

    return RSVDFunction


_RSVD_FN = None


def svd_autograd(A, plan):
    """Differentiable rank-k randomized SVD through the library: returns (U, S, V) whose
    gradients flow to the float32 tensor A through rsvd_svd_backward.  The plan's last
    rsvd_svd must be this call's when backward runs (one forward per backward)."""
    global _RSVD_FN
    if _RSVD_FN is None:
        _RSVD_FN = _autograd_function()
    return _RSVD_FN.apply(A, plan)


def split_bf16(A):
    """float32 CUDA tensor (m x n) -> bfloat16 (2m x n): hi = bf16(A) over lo = bf16(A - hi),
    the RSVD_BF16X2 layout (computed by the library's conversion kernel)."""
    import torch

    m, n = A.shape
    out = torch.empty(2 * m, n, device=A.device, dtype=torch.bfloat16)
    rsvd_convert_a(A, m, n, A.stride(0), out, n, 1)
    return out


def svd(A, k, p=10, q=1, seed=0, precision=None, orth_rounds=3):
    """Rank-k randomized SVD of a CUDA tensor A (float32 -> plain FP32 path,
    bfloat16 -> tensor-core path).  Returns float32 (U, S, V)."""
    import torch

    if precision is None:
        precision = RSVD_BF16_TC if A.dtype == torch.bfloat16 else RSVD_PLAIN_FP32
    m, n = A.shape
    with Plan(m, n, k, p, q, seed, precision, orth_rounds, lda=A.stride(0)) as pl:
        return pl.svd(A)


class BatchedPlan:
    """Randomized SVD of many small bfloat16 matrices (l = k + p <= 32) with one plan.

    shapes: list of (m_b, n_b); lda_b defaults to n_b rounded up to 8.  Outputs are
    concatenated: U (sum m_b, k), S (batch, k), V (sum n_b, k)."""

    def __init__(self, shapes, k, p=8, q=1, seed=0, lda=None, stream=None, orth_rounds=3,
                 autotune=1):
        self.shapes = [(int(a), int(b)) for a, b in shapes]
        self.batch = len(self.shapes)
        self.k, self.p, self.q = int(k), int(p), int(q)
        ms = (ctypes.c_int64 * self.batch)(*[a for a, _ in self.shapes])
        ns = (ctypes.c_int64 * self.batch)(*[b for _, b in self.shapes])
        ld = None if lda is None else (ctypes.c_int64 * self.batch)(*[int(x) for x in lda])
        o = rsvd_options_default()
        o.precision = RSVD_BF16_TC
        o.dtype_A = RSVD_BF16
        o.orth_rounds = orth_rounds
        o.autotune = autotune
        h = ctypes.c_void_p()
        _check(lib().rsvd_batched_plan_create(ctypes.byref(h), self.batch, ms, ns, ld, self.k, self.p,
                                              self.q, int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.byref(o),
                                              _stream(stream)), "rsvd_batched_plan_create")
        self.handle = h.value
        self.row_m = [0]
        self.row_n = [0]
        for a, b in self.shapes:
            self.row_m.append(self.row_m[-1] + a)
            self.row_n.append(self.row_n[-1] + b)

    def close(self):
        if self.handle is not None:
            lib().rsvd_batched_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def svd(self, mats, U=None, S=None, V=None):
        import torch

        ptrs = (ctypes.c_void_p * self.batch)(*[int(a.data_ptr()) for a in mats])
        dev = mats[0].device
        if U is None:
            U = torch.empty(self.row_m[-1], self.k, device=dev)
            S = torch.empty(self.batch, self.k, device=dev)
            V = torch.empty(self.row_n[-1], self.k, device=dev)
        _check(lib().rsvd_batched_svd(self.handle, ptrs, _ptr(U), _ptr(S), _ptr(V)), "rsvd_batched_svd")
        self._keep = ptrs
        return U, S, V

    def backward(self, mats, grads=None):
        """dL/dA_b for the matrices of the last svd() call; grads: float32 (m_b, n_b) tensors."""
        import torch

        if grads is None:
            grads = [torch.empty(a, b, device=mats[0].device) for a, b in self.shapes]
        ptrs = (ctypes.c_void_p * self.batch)(*[int(a.data_ptr()) for a in mats])
        gptrs = (ctypes.c_void_p * self.batch)(*[int(g.data_ptr()) for g in grads])
        _check(lib().rsvd_batched_svd_backward(self.handle, ptrs, gptrs), "rsvd_batched_svd_backward")
        self._keep_b = (ptrs, gptrs)
        return grads

    def tuning(self):
        """{'stages': [4], 'ctas_per_sm': [4], 'tuned': bool} of the grouped pass (per
        pass kind 2 mode + fold)."""
        st = (ctypes.c_int32 * 4)()
        ct = (ctypes.c_int32 * 4)()
        tu = ctypes.c_int32(0)
        _check(lib().rsvd_batched_tuning(self.handle, st, ct, ctypes.byref(tu)), "rsvd_batched_tuning")
        return {"stages": list(st), "ctas_per_sm": list(ct), "tuned": bool(tu.value)}

    def sync(self):
        sw = ctypes.c_uint32(0)
        _check(lib().rsvd_batched_sync(self.handle, ctypes.byref(sw)), "rsvd_batched_sync")
        return int(sw.value)
