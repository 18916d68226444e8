/*
 * rsvd.h -- C ABI of the GB300 (sm_103a) randomized range finder and
 * randomized SVD library.
 *
 * The computation follows Halko, Martinsson and Tropp, "Finding structure with
 * randomness" (SIAM Review 53(2), 2011):
 *   Stage A: draw a test matrix Omega (Algorithm 4.1 step 1; the SRFT of
 *            Section 4.6), form Y = A Omega, and run q steps of randomized
 *            subspace iteration (Algorithm 4.4), orthonormalising after every
 *            application of A or A^T (the round-off remark of Section 4.5);
 *   Stage B: form B = Q^T A, take the SVD of the small matrix and lift
 *            U = Q Ut (Algorithm 5.1), truncated to rank k (Remark 5.1).
 * The problem solved is the fixed-rank problem of Section 1.3: a target rank
 * k and an oversampling p give a basis of l = k + p columns.
 *
 * Conventions for every entry point:
 *   - Matrices are row-major.  A is m x n with leading dimension lda >= n
 *     (elements), float32 or bfloat16 as chosen in rsvd_options_t.
 *   - Pointers named *_host are host memory; every other matrix pointer is
 *     device memory on the current CUDA device.  The caller owns all of them.
 *   - "stream" arguments are cudaStream_t values passed as void* (NULL = the
 *     legacy default stream).  Work is enqueued asynchronously on the plan's
 *     stream; argument errors are returned at once, errors found on the
 *     device (breakdown, non-finite data, a bounded wait that expired) are
 *     recorded in the plan's device status word and returned by rsvd_sync()
 *     and by the next call on the plan.
 *   - A plan is not thread safe; distinct plans may be used concurrently.
 *   - Singular values are returned in descending order.  The sign of each
 *     singular-vector pair (u_j, v_j) is not specified.
 */
#ifndef PAPER_0909_4061_RSVD_H
#define PAPER_0909_4061_RSVD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RSVD_API __attribute__((visibility("default")))
#else
#define RSVD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rsvd_plan_s* rsvd_plan_t;

typedef enum {
  RSVD_OK = 0,
  RSVD_ERR_INVALID_ARG = 1,   /* bad sizes, null pointers, misaligned lda, unsupported combination */
  RSVD_ERR_ALLOC = 2,         /* device or pinned-host allocation failed */
  RSVD_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  RSVD_ERR_NUMERICAL = 4,     /* Cholesky or Jacobi breakdown that the safeguards could not absorb */
  RSVD_ERR_NONFINITE = 5,     /* NaN or Inf met in A or in an intermediate */
  RSVD_ERR_TIMEOUT = 6,       /* a bounded device-side wait expired */
  RSVD_ERR_UNSUPPORTED = 7    /* valid request the library does not implement (yet) */
} rsvd_status_t;

/* element type of A.  RSVD_BF16X2: A is stored as two bfloat16 m x n blocks with the
 * same lda, the rounded values hi = bf16(A) followed (m * lda elements further) by the
 * residual lo = bf16(A - hi), as rsvd_convert_a writes them; the final pass B^T = A^T Q
 * reads both (about 16 significant bits), and with residual_passes = 1 every pass does. */
enum { RSVD_F32 = 0, RSVD_BF16 = 1, RSVD_BF16X2 = 2 };
enum { RSVD_GAUSSIAN = 0, RSVD_SRFT = 1, RSVD_GSRFT = 2 };  /* test matrix (Section 4.1 / 4.6) */
enum { RSVD_PLAIN_FP32 = 0, RSVD_BF16_TC = 1 };       /* how the passes over A are computed */

typedef struct {
  int32_t dtype_A;      /* RSVD_F32, RSVD_BF16 or RSVD_BF16X2 */
  int32_t test_matrix;  /* RSVD_GAUSSIAN (default) or RSVD_SRFT: sqrt(n/l_c) D F R with
                           random +-1 signs D, the unitary DFT F and l_c = l / 2 frequencies
                           from {1 .. n/2 - 1} without replacement; for a real A the l real
                           columns are [Re, Im] of each sampled frequency.  Needs l and n
                           even and n < 2^24.  RSVD_GSRFT: the modified SRFT of Section 4.6
                           (eq. random_Givens), D'' Theta' D' Theta times that SRFT, Theta =
                           Pi G(1,2; t_1) ... G(n-1,n; t_{n-1}) a random permutation after a
                           chain of random real Givens rotations, D', D'' random signs; the
                           same size rules */
  int32_t precision;    /* RSVD_PLAIN_FP32: float32 A, float32 FMA on CUDA cores.
                           RSVD_BF16_TC: bfloat16 A (RSVD_BF16 or RSVD_BF16X2), tcgen05
                           tensor-core products with float32 accumulation, float32
                           re-orthonormalisation, and a split (hi + lo) basis in the final
                           pass B^T = A^T Q (with RSVD_BF16X2 also a split A there, or in
                           every pass with residual_passes = 1). */
  int32_t single_pass;  /* 1: two-sided one-pass sketch of Section 5.5 (q ignored) */
  int32_t recompute;    /* backward: recompute the sample matrices instead of storing them */
  int32_t orth_rounds;  /* Cholesky-QR rounds per orthonormalisation of a final basis: 2 or
                           3 (default 3: one shifted round for ill-conditioned samples, then
                           two plain); the intermediate bases of the power iteration get at
                           most 2 (the shifted round and one plain one) */
  int64_t lda;          /* leading dimension of A in elements; 0 means n */
  int32_t small_svd;    /* kernel of the l x l SVD (Algorithm 5.1 step 2): RSVD_SMALL_AUTO
                           (default), RSVD_SMALL_ONE_CTA (l <= 160) or RSVD_SMALL_CLUSTER
                           (a thread-block cluster of 4 or 8 CTAs, l <= 256); AUTO takes the
                           cluster from l = 48 on */
  int32_t residual_passes; /* with dtype_A RSVD_BF16X2: 0 (default) only the final pass
                           reads hi + lo; 1 every pass over A does (twice the bytes of A per
                           pass; the reconstruction error then matches the float32 path's to
                           about 1e-5 relative where a hi-only Stage A leaves 2e-4 to 1e-3);
                           2 the passes whose samples become final bases do (the last pass
                           of Stage A, Y = A Qt_q or Y = A Omega for q = 0, the single pass's
                           sketches, rsvd_sketch) besides the final one, the earlier power-
                           iteration passes read hi only (between the two: the float64 model
                           puts its excess at up to 6e-4 at 2048 x 2048, q = 1, against
                           4e-5 for every pass).  Must be 0 for other dtypes */
  int32_t psi_cols;     /* single pass: columns l' of the second test matrix Psi (m x l'),
                           k <= l' <= min(n, 256); 0 (default) takes min(3 l, 256, n).  A Psi
                           wider than l makes the system for B^T overdetermined (Section 5.5,
                           the remark on single-pass error) */
  int32_t srft_fft;     /* SRFT plans: 1 forms the first pass Y = A Omega by the transform
                           along the rows of A (rsvd_sketch_srft; no n x l matrix), 0
                           (default) by a tensor-core (or float32) pass with the drawn
                           n x l matrix, which is faster on this GPU at l <= 256 */
  int32_t autotune;     /* batched plans: 1 (default) times the grouped pass's configurations
                           (pipeline stages x CTAs per SM) on the first rsvd_batched_svd call
                           and keeps the fastest per pass kind, cached per shape class in
                           the JSON file named by the environment variable RSVD_TUNE_CACHE
                           when it is set; 0 keeps the built-in configuration */
  int32_t host_f32;     /* 1: rsvd_svd_host takes A as float32 (m x n, leading dimension
                           lda) and converts it on the device to the plan's bfloat16 storage
                           (hi, and lo for RSVD_BF16X2) before the SVD, so a caller holding a
                           float32 matrix needs no conversion of its own.  Only with
                           RSVD_BF16_TC; 0 (default): A_host is in the plan's dtype */
} rsvd_options_t;

enum { RSVD_SMALL_AUTO = 0, RSVD_SMALL_ONE_CTA = 1, RSVD_SMALL_CLUSTER = 2 };

/* Fill *opt with the defaults: float32 A, Gaussian test matrix, plain FP32,
 * two-pass Stage B, three orthonormalisation rounds, lda = n. */
RSVD_API void rsvd_options_default(rsvd_options_t* opt);

/* Create a plan for the fixed-rank problem (Section 1.3): A is m x n, target
 * rank k >= 1, oversampling p >= 0, q >= 0 power steps (Algorithm 4.4), and
 * the test-matrix seed.  Requires l = k + p <= min(m, n) and l <= 256.  All
 * device workspace is allocated here (rsvd_workspace_bytes reports it); the
 * plan's work runs on `stream`.  On failure *plan is set to NULL. */
RSVD_API rsvd_status_t rsvd_plan_create(rsvd_plan_t* plan, int64_t m, int64_t n, int32_t k,
                               int32_t p, int32_t q, uint64_t seed,
                               const rsvd_options_t* opt, void* stream);

/* Release the plan and its workspace (waits for its stream first).  NULL is a no-op. */
RSVD_API rsvd_status_t rsvd_plan_destroy(rsvd_plan_t plan);

/* Device workspace held by the plan, in bytes. */
RSVD_API rsvd_status_t rsvd_workspace_bytes(rsvd_plan_t plan, size_t* bytes);

/* Stage A only (Algorithm 4.4; Algorithm 4.1 when q = 0; Algorithm 4.5 for the
 * SRFT).  A: device, m x n.  Q: device, m x l float32 with leading dimension
 * ldq >= l; on return its columns are an orthonormal basis approximating the
 * range of A, in the order the orthonormaliser produces them (diag(R) > 0). */
RSVD_API rsvd_status_t rsvd_range_finder(rsvd_plan_t plan, const void* A, float* Q, int64_t ldq);

/* Stage A + Stage B (Algorithm 4.4 then Algorithm 5.1 with the Remark 5.1
 * truncation).  A: device, m x n.  U: device m x k, S: device k, V: device
 * n x k, all float32 row-major with leading dimension k.  A ~= U diag(S) V^T. */
RSVD_API rsvd_status_t rsvd_svd(rsvd_plan_t plan, const void* A, float* U, float* S, float* V);

/* The interpolative decomposition of the rows of Y (Section 3.2.3): an index set J of l
 * rows and X (m x l) with X[J, :] = I and Y = X Y[J, :], for Y of rank l.  The rows are
 * chosen by successive orthogonalization with pivoting (Businger--Golub, Section 3.3.2,
 * applied to the rows: at each step the row with the longest residual; ties to the lowest
 * index), one cooperative launch of one CTA per SM with a grid barrier per step; X =
 * C L^-1 from the coefficients C of every row on the pivot directions and their
 * triangular block L = C[J, :].
 *   Y: device, m x l float32 (the plan's m and l), leading dimension ldy >= l; read only.
 *   J: device, l int32, the pivots in the order chosen; X: device, m x l float32, ldx >= l.
 * Y of rank < l: the pivots from the step where no row is left are -1 and rsvd_sync
 * returns RSVD_ERR_NUMERICAL.  The entries of X are not bounded by 2 in general (that
 * bound belongs to the strong rank-revealing ID); they are small for bases from Stage A. */
RSVD_API rsvd_status_t rsvd_row_id(rsvd_plan_t plan, const float* Y, int64_t ldy, int32_t* J,
                                   float* X, int64_t ldx);

/* Stage B by row extraction (Algorithm 5.2) after Stage A as in rsvd_svd: the ID of the
 * basis, Q = X Q[J, :] (rsvd_row_id); A[J, :]^T = W R (Cholesky-QR); Z = X R^T; Z = U S Vt^T
 * (Cholesky-QR and Jacobi); V = W Vt.  A is read by Stage A and in l rows only: no pass
 * B = Q^T A.  ||A - U S V^T|| <= (1 + ||X||) ||A - Q Q^T A|| (Lemma 5.1), usually larger
 * than the error of rsvd_svd.  Outputs as rsvd_svd (device U m x k, S k, V n x k). */
RSVD_API rsvd_status_t rsvd_svd_row_extraction(rsvd_plan_t plan, const void* A, float* U, float* S,
                                               float* V);

/* Stage B for a symmetric A (m = n; Section 5.3, 5.4), after Stage A as in rsvd_svd:
 *   RSVD_EIG_DIRECT  -- Algorithm 5.3: B = Q^T A Q, B = V Lambda V^T, U = Q V
 *                       (||A - U Lambda U^T|| <= 2 ||A - Q Q^T A||);
 *   RSVD_EIG_NYSTROM -- Algorithm 5.5 for a positive semidefinite A: B1 = A Q,
 *                       Q^T B1 = C^T C (Cholesky), F = B1 C^-1, F = U S W^T, Lambda = S^2
 *                       (A ~ F F^T, never worse than ||A - Q Q^T A|| in the spectral norm).
 * A is read once more than by the range finder (B1 = A Q).  Outputs: U (device, m x k
 * float32, leading dimension k) and Lambda (device, k), the k eigenvalues of largest
 * magnitude in decreasing order of |lambda|; the sign of each eigenvector is not
 * specified.  The symmetry of A is assumed, not checked. */
enum { RSVD_EIG_DIRECT = 0, RSVD_EIG_NYSTROM = 1 };
RSVD_API rsvd_status_t rsvd_eig(rsvd_plan_t plan, const void* A, int32_t method, float* U,
                                float* Lambda);

/* The fixed-precision problem (Section 4.4): Algorithm 4.2, the adaptive randomized range
 * finder, in the blocked form of the remark that follows it.  Samples A w_i (the Gaussian
 * columns of Philox stream 3 for the plan's seed) are taken `block` at a time; each block's
 * posterior estimate max_i ||(I - Q Q^T) A w_i|| (Lemma 4.1, estimate (4.3)) is compared
 * with eps / (10 sqrt(2/pi)); while it is larger the block is reprojected, orthonormalised,
 * reprojected once normalised, orthonormalised again and appended to Q, and the next block
 * is sampled.  On return ||(I - Q Q^T) A|| <= eps except with probability
 * min(m, n) 10^-block, unless the basis reached its cap first.
 *   The plan sets the cap: at most l = k + p columns (q is not used).  block: a multiple of
 *   16, 16 <= block <= l.  Q: device, m x l float32, leading dimension ldq >= l; its first
 *   *rank columns (a multiple of block) are the basis.  *estimate (may be NULL) receives
 *   the last block's estimate.  The call waits for the device once per block (the host
 *   takes the stopping decision). */
RSVD_API rsvd_status_t rsvd_range_finder_adaptive(rsvd_plan_t plan, const void* A, float eps,
                                                  int32_t block, float* Q, int64_t ldq,
                                                  int32_t* rank, float* estimate);

/* rsvd_svd for host-resident data: copies A (host, m x n with the plan's lda,
 * in the plan's dtype, or float32 with the host_f32 option) to a device buffer
 * owned by the plan (allocated on the first call; the copy goes in four pieces on four
 * streams of the plan), runs rsvd_svd,
 * copies U, S, V back to host memory, and waits for completion.  Page-locked host
 * buffers give the full copy bandwidth; pageable buffers work but are staged by the
 * driver. */
RSVD_API rsvd_status_t rsvd_svd_host(rsvd_plan_t plan, const void* A_host, float* U_host,
                            float* S_host, float* V_host);

/* Gradient of L = ||A - U diag(S) V^T||_F^2 + sum(S) composed with the
 * caller's loss, Omega held fixed: given the cotangents gU (m x k), gS (k),
 * gV (n x k) of the caller's loss (any may be NULL = zero) plus the built-in
 * reconstruction term when add_recon != 0, writes gA (device, m x n float32,
 * leading dimension n).  Must follow an rsvd_svd call on the same A. */
RSVD_API rsvd_status_t rsvd_svd_backward(rsvd_plan_t plan, const void* A, const float* gU,
                                const float* gS, const float* gV, int32_t add_recon,
                                float* gA);

/* Parity hooks for the test matrix.  get: copy the plan's n x l Omega (device
 * float32, leading dimension l) as drawn for its seed or as last set.  set:
 * use the caller's n x l Omega (device float32, leading dimension l) instead
 * of the seeded draw; NULL returns to the seeded draw. */
RSVD_API rsvd_status_t rsvd_get_omega(rsvd_plan_t plan, float* Omega);
RSVD_API rsvd_status_t rsvd_set_omega(rsvd_plan_t plan, const float* Omega);

/* Wait for the plan's stream and return the first device-detected error
 * since the previous rsvd_sync (RSVD_OK if none); clears it. */
RSVD_API rsvd_status_t rsvd_sync(rsvd_plan_t plan);

/* ---- failure detection, tested without a fault --------------------------
 * Every device-side wait of the library (mbarrier phases, stream-K hand-over flags) is
 * bounded: when it runs out the kernel records RSVD_ERR_TIMEOUT in the plan's status word,
 * lets its own copies in flight land, releases its tensor memory and returns, so the
 * CUDA context stays usable and rsvd_sync() reports the timeout. */

/* Diagnostic of that path: enqueues on the plan's stream a kernel that waits for a device
 * word nothing ever sets, with a limit of `spins` polls about 64 ns apart (spins >= 1);
 * the wait always runs out, the kernel records the timeout and returns, and the next
 * rsvd_sync() returns RSVD_ERR_TIMEOUT (and clears it).  The paper has no counterpart. */
RSVD_API rsvd_status_t rsvd_wait_selftest(rsvd_plan_t plan, uint32_t spins);

/* Failure injection for tests of allocation-failure handling: the `after`-th device
 * allocation the library makes from now on (0 = the next one) fails as a failed
 * cudaMalloc would, with RSVD_ERR_ALLOC and no workspace leaked; -1 disarms.  The setting
 * is process wide and is consumed by the failure.  The paper has no counterpart. */
RSVD_API void rsvd_debug_fail_alloc(int32_t after);

/* Static English description of a status code. */
RSVD_API const char* rsvd_status_string(rsvd_status_t status);

/* ---- tracing ----------------------------------------------------------- */

/* Diagnostics of the device-side work since the previous call (waits for the
 * plan's stream): out[0] = status bits seen, including the informational ones
 * (4: a Cholesky pivot was replaced by the floor because the sample is
 * numerically rank deficient; 16: the Jacobi sweeps hit their limit); out[1] =
 * the largest number of Jacobi sweeps taken by one small SVD.  n is the length
 * of out (<= 2 entries are written); out[1] is reset. */
RSVD_API rsvd_status_t rsvd_diagnostics(rsvd_plan_t plan, uint32_t* out, int32_t n);

/* Step kinds for per-step timing and launch counts. */
enum {
  RSVD_STEP_DRAW = 0,       /* test matrix (Algorithm 4.1 step 1) */
  RSVD_STEP_PASS = 1,       /* one pass over A: Y = A X or A^T X */
  RSVD_STEP_ORTH = 2,       /* Cholesky-QR rounds (Gram, factor, apply) */
  RSVD_STEP_SMALL_SVD = 3,  /* Jacobi SVD of the l x l factor */
  RSVD_STEP_LIFT = 4,       /* U = Q Ut_k, V = Q_B W_k */
  RSVD_STEP_CONVERT = 5,    /* float32 -> transposed bfloat16 operands */
  RSVD_STEP_ID = 6,         /* pivoted row selection of the interpolative decomposition */
  RSVD_NUM_STEPS = 7
};

/* Start per-step timing: for every step kind whose bit is set in `mask`,
 * each later step of that kind on this plan is bracketed by a pair of CUDA
 * events recorded on the plan's stream.  Resets the time totals and the
 * kernel launch counters (which are kept for every kind, whatever the mask).
 * mask = 0 stops timing. */
RSVD_API rsvd_status_t rsvd_profile(rsvd_plan_t plan, uint32_t mask);

/* Waits for the plan's stream, then for each step kind s < nkinds writes the
 * summed device time of the timed steps (ms[s], milliseconds; may be NULL)
 * and the number of kernels launched (launches[s]; may be NULL) since the
 * last rsvd_profile call. */
RSVD_API rsvd_status_t rsvd_profile_read(rsvd_plan_t plan, float* ms, int64_t* launches,
                                         int32_t nkinds);

/* ---- step-level entry points (each runs one step of the method with the
 * ---- plan's kernels; the tests check each against the oracle) ---------- */

/* Input staging for the tensor-core path (not part of a timed SVD): A (device
 * float32, m x n, lda) -> out (device bfloat16, leading dimension ldo): hi = bf16(A)
 * in the first m rows and, when with_lo != 0, lo = bf16(A - hi) in the next m rows
 * (the RSVD_BF16X2 layout; out must hold 2 m rows then). */
RSVD_API rsvd_status_t rsvd_convert_a(const float* A, int64_t m, int64_t n, int64_t lda,
                                      void* out, int64_t ldo, int32_t with_lo, void* stream);

/* Algorithm 4.1 step 1: rows x cols standard Gaussian matrix into `out`
 * (device float32, leading dimension ld >= cols).  Element (i, j): with
 * g = j / 4, t = j % 4, the Philox4x32-10 block for counter (g, i, stream_id, 0)
 * and key (seed mod 2^32, seed / 2^32) gives words x0..x3; u_a =
 * (2 (x_a >> 9) + 1) 2^-24; z0, z1 = sqrt(-2 ln u0) (cos, sin)(2 pi u1) and
 * z2, z3 likewise from (u2, u3); the element is z_t. */
RSVD_API rsvd_status_t rsvd_draw_gaussian(uint64_t seed, uint32_t stream_id, int64_t rows,
                                 int64_t cols, float* out, int64_t ld, void* stream);

/* One pass over A with the plan's precision: transpose = 0 gives Y = A X
 * (X: n x l, Y: m x l); transpose = 1 gives Y = A^T X (X: m x l, Y: n x l).
 * X and Y are device float32 with leading dimension l. */
RSVD_API rsvd_status_t rsvd_sketch(rsvd_plan_t plan, const void* A, int32_t transpose,
                          const float* X, float* Y);

/* The first pass of an SRFT plan, Y = A Omega (m x l, device float32, leading dimension l),
 * computed as the paper's transform along the rows of A (Algorithm 4.5 step 2; Section
 * 4.6): for every row, the random signs, a length-n FFT in shared memory (n / 2 complex
 * points, four-step), and the l / 2 sampled frequencies as [Re, Im] columns scaled by
 * (l / 2)^-1/2 -- no n x l matrix is formed.  It applies for n a power of two in
 * [2048, 32768] and an even lda (else RSVD_ERR_UNSUPPORTED); rsvd_svd and
 * rsvd_range_finder take this route for their first pass when the plan has srft_fft = 1
 * and its own draw (after rsvd_set_omega the given matrix is multiplied instead). */
RSVD_API rsvd_status_t rsvd_sketch_srft(rsvd_plan_t plan, const void* A, float* Y);

/* Orthonormalise the columns of Y (device float32, rows x l, leading
 * dimension l, rows <= max(m, n)) in place with the plan's Cholesky-QR
 * rounds; R (device float32, l x l, may be NULL) receives the upper
 * triangular factor with Y_in = Y_out R. */
RSVD_API rsvd_status_t rsvd_orthonormalize(rsvd_plan_t plan, int64_t rows, float* Y, float* R);

/* SVD of a small l x l matrix X (device float32, leading dimension l):
 * X = Ut diag(S) W^T with Ut, W (device, l x l, leading dimension l) and S
 * (device, l) descending, by one-sided Jacobi rotations. */
RSVD_API rsvd_status_t rsvd_small_svd(rsvd_plan_t plan, const float* X, float* Ut, float* S,
                             float* W);

/* ---- allocation-free pass ------------------------------------------------ */

/* One tensor-core pass over a bfloat16 A without allocating any memory:
 * Y = A X (transpose = 0) or Y = A^T X (transpose = 1).  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- a service whose device memory is carved up once at start-up by
 * its own allocator, code that runs while a stream is being captured into a
 * CUDA graph, or a latency-critical loop where cudaMalloc's implicit device
 * synchronisation is not acceptable.  It needs no plan.
 *
 *   A:  device bfloat16, m x n row-major, leading dimension lda (multiple of 8,
 *       16-byte-aligned base).
 *   Xt: device bfloat16, the operand stored transposed: l rows of K elements
 *       (K = n when transpose = 0, m when transpose = 1), leading dimension
 *       ldxt >= K, a multiple of 8, 16-byte-aligned base.
 *   l:  a multiple of 16, 16 <= l <= 128.
 *   Y:  device float32, (transpose ? n : m) x l row-major, leading dimension l,
 *       16-byte-aligned base (the results are stored four floats at a time).
 *   status: device word that receives a timeout bit (8) if a bounded wait
 *       expires; may be NULL.
 * Sizes outside these limits return RSVD_ERR_INVALID_ARG before any work.
 *
 * The scratch it needs (partial sums of output row tiles shared by two CTAs
 * and their hand-over flags) is a fixed static device array of 152 x 128 x
 * 128 floats (9.5 MiB) plus 152 words, held by every GPU that loads the
 * library until the process exits.  The first call on a device sets it up
 * (looks up the array's device address and the kernel's shared-memory limit),
 * so make that first call before any stream capture.  Every call shares the
 * array: calls whose kernels overlap on the GPU (other streams, other threads)
 * race on it and give wrong results; order them on one stream.  The call is
 * asynchronous on `stream`. */
RSVD_API rsvd_status_t rsvd_sketch_bf16_noalloc(const void* A, int64_t m, int64_t n,
                                                int64_t lda, int32_t transpose, const void* Xt,
                                                int64_t ldxt, int32_t l, float* Y,
                                                uint32_t* status, void* stream);

/* ---- Batched: many small matrices, one plan --------------------------------
 * The randomized SVD of Algorithm 4.4 + Algorithm 5.1 (with the Gaussian test
 * matrix of Algorithm 4.1) applied to `batch` independent matrices A_b, every step
 * one launch over the whole batch: grouped tensor-core passes (bfloat16 A_b,
 * float32 accumulation), one CTA per matrix for the Cholesky-QR rounds and for the
 * l x l one-sided Jacobi SVD.  Requires l = k + p <= 32, m_b >= l, n_b >= l,
 * precision RSVD_BF16_TC with dtype_A RSVD_BF16, the Gaussian test matrix; anything
 * else returns RSVD_ERR_UNSUPPORTED (or RSVD_ERR_INVALID_ARG for bad sizes).
 * Omega_b is drawn from seed + b (Philox4x32-10, stream 0, as rsvd_draw_gaussian).
 * m, n (and lda, or NULL for lda_b = n_b rounded up to 8; each lda_b a multiple of 8)
 * are host arrays of `batch` entries, copied at creation.  The plan is not thread-safe. */
typedef struct rsvd_batched_plan_s* rsvd_batched_plan_t;

RSVD_API rsvd_status_t rsvd_batched_plan_create(rsvd_batched_plan_t* plan, int32_t batch,
                                                const int64_t* m, const int64_t* n,
                                                const int64_t* lda, int32_t k, int32_t p,
                                                int32_t q, uint64_t seed,
                                                const rsvd_options_t* opt, void* stream);
RSVD_API rsvd_status_t rsvd_batched_plan_destroy(rsvd_batched_plan_t plan);

/* A: host array of `batch` device pointers (bfloat16, m_b x n_b row-major, lda_b,
 * 16-byte-aligned).  Outputs, device float32: U is sum(m_b) x k with matrix b's rows
 * from row sum_{c<b} m_c; S is batch x k (descending per matrix); V is sum(n_b) x k
 * likewise.  Asynchronous on the plan's stream; the plan keeps what the backward
 * pass needs (the bases, R factors and small SVDs of this call). */
RSVD_API rsvd_status_t rsvd_batched_svd(rsvd_batched_plan_t plan, const void* const* A, float* U,
                                        float* S, float* V);

/* Gradient of L = sum_b ||A_b - U_b S_b V_b^T||_F^2 + sum_b sum_{i<=k} sigma_{b,i} with
 * respect to every A_b, through the map of rsvd_batched_svd with the test matrices
 * held fixed (reverse mode through the passes, the Cholesky-QR steps and the SVD of
 * B; no counterpart in the paper, which does not differentiate its algorithms).  A
 * must be the matrices of the plan's last rsvd_batched_svd call (its bases and
 * factors are reused).  gA: host array of `batch` device pointers to float32
 * m_b x n_b row-major (leading dimension n_b) outputs.  It reads A 2q + 2 times
 * more and writes every gA_b once; asynchronous on the plan's stream. */
RSVD_API rsvd_status_t rsvd_batched_svd_backward(rsvd_batched_plan_t plan, const void* const* A,
                                                 float* const* gA);

/* The grouped pass's configuration in use, per pass kind c = 2 mode + fold (mode 0: Y = A X,
 * 1: Y = A^T X; fold: the operand carries a lo half): stages[c] pipeline stages and ctas[c]
 * CTAs per SM (4 entries each; either may be NULL).  *tuned = 1 once the autotuner has
 * chosen them (may be NULL). */
RSVD_API rsvd_status_t rsvd_batched_tuning(rsvd_batched_plan_t plan, int32_t* stages, int32_t* ctas,
                                           int32_t* tuned);

/* Waits for the plan's stream and returns the device status as rsvd_sync does;
 * *sweeps (may be NULL) receives the largest Jacobi sweep count since the last call. */
RSVD_API rsvd_status_t rsvd_batched_sync(rsvd_batched_plan_t plan, uint32_t* sweeps);

#ifdef __cplusplus
}
#endif

#endif /* PAPER_0909_4061_RSVD_H */
