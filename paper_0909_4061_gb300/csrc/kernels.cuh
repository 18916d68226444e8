// Launchers of the library's kernels (host side).  Every step of the path
// runs in one of these kernels; the C ABI in api.cu only sequences them.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rsvd {

// Algorithm 4.1 step 1: rows x cols Gaussian, columns [cols, cols_pad) zero.
// out (float32, ld) and/or out_t (bfloat16 transposed, cols_pad x rows, ld_t) may be null.
cudaError_t launch_draw_gaussian(uint64_t seed, uint32_t stream_id, int64_t rows, int cols,
                                 int cols_pad, float* out, int64_t ld, __nv_bfloat16* out_t,
                                 int64_t ld_t, cudaStream_t st);

// C[s] = op(A)[:, Ks] * X[Ks, :] over split s of the K range, float32 FMA.
// trans = 0: op(A) = A (M x K, lda); trans = 1: op(A) = A^T with A stored K x M (lda).
// X is K x N (ldx), C is M x N (ldc); split s writes C + s * split_stride.
cudaError_t launch_gemm_f32(int trans, int64_t M, int64_t N, int64_t K, const float* A,
                            int64_t lda, const float* X, int64_t ldx, float* C, int64_t ldc,
                            int splits, int64_t split_stride, cudaStream_t st);

// Partial Gram matrices of the rows of Y (rows x lp, ld lp) over nblk row blocks;
// when splits > 1, Y is first formed as the sum of `splits` partial slabs
// (src + s * split_stride) and written to y_out.
cudaError_t launch_gram_partial(const float* src, int splits, int64_t split_stride, float* y_out,
                                int64_t rows, int lp, float* gpart, int nblk, cudaStream_t st);
int gram_blocks(int64_t rows);

// The same partials on the tensor cores (each entry of Y split exactly into three bfloat16
// parts, six products, float32 accumulation) over gram_tc_grid(rows, nblk_max) row blocks,
// lower triangles only; lp a multiple of 16 up to 256.
int gram_tc_grid(int64_t rows, int nblk_max);
cudaError_t launch_gram_tc(const float* src, int splits, int64_t split_stride, float* y_out,
                           int64_t rows, int lp, float* gpart, int nblk, uint32_t* status,
                           cudaStream_t st);

// Q = Y R^-1 on the tensor cores (Y and R^-1 split exactly into three bfloat16 parts, six
// products): img (apply_tc_image_bytes(lp) bytes) receives the planes of R^-1 first.
size_t apply_tc_image_bytes(int lp);
cudaError_t launch_apply_tc(const float* y, float* q, int64_t rows, int lp, const float* rinv,
                            void* img, uint32_t* status, cudaStream_t st);

// G = sum of the nblk partial Grams (lp x lp).
cudaError_t launch_gram_reduce(const float* gpart, int nblk, int lp, float* g, cudaStream_t st);

// Q = Y R^-1 (rows x lp, lp a multiple of 16 up to 128, R^-1 upper triangular, nblk row
// blocks) and, with do_gram, the lower triangle of each block's Gram partial Q^T Q into
// gpart (nblk x lp x lp) for launch_gram_reduce.
cudaError_t launch_apply_gram(const float* y, float* q, int64_t rows, int lp, const float* rinv,
                              float* gpart, int nblk, int do_gram, cudaStream_t st);
// The lower triangle of the Gram partials of Y (the sum of `splits` slabs, written to y_out
// when y_out is non-null) for the same lp range.
cudaError_t launch_gram_tri(const float* src, int splits, int64_t split_stride, float* y_out,
                            int64_t rows, int lp, float* gpart, int nblk, cudaStream_t st);

// Cholesky G (+ shift) = R^T R, R^-1 into rinv (lp x lp upper, zero padded), R into r_out,
// and racc <- R * racc (or racc <- R when racc_init != 0) when racc is non-null.
cudaError_t launch_cholesky(const float* g, int l, int lp, int shifted, float* lbuf, float* r_out,
                            float* rinv, float* racc, int racc_init, uint32_t* status,
                            cudaStream_t st);

// float32 rows x lp (ld lp) -> bfloat16 transposed (lp x rows, ld_t); with `split`,
// also writes the residual x - bf16(x) as rows [lo_off, lo_off + lp) of the output.
cudaError_t launch_to_bf16_t(const float* x, int64_t rows, int lp, __nv_bfloat16* out,
                             int64_t ld_t, int split, int lo_off, cudaStream_t st);

// A (float32, rows x cols, ld) -> bfloat16 hi (rows x cols, ld_out) and, with_lo, the
// bfloat16 residual lo = bf16(A - hi) lo_off elements further (default, lo_off < 0: the
// rows x cols block that follows, rows * ld_out elements further).
cudaError_t launch_split_bf16(const float* x, int64_t rows, int64_t cols, int64_t ld,
                              __nv_bfloat16* out, int64_t ld_out, int with_lo, cudaStream_t st,
                              int64_t lo_off = -1);

// float32 <-> bfloat16 conversion of a whole matrix (rows x cols, ld) for A.
cudaError_t launch_f32_to_bf16(const float* x, int64_t rows, int64_t cols, int64_t ld,
                               __nv_bfloat16* out, int64_t ld_out, cudaStream_t st);

// One-sided Jacobi SVD of X = R^T (transposed = 1, R row-major l x l, ld) or X (transposed = 0).
// Outputs: ut (l x l, ld lp), s (l), w (l x l, ld lp), descending.
// info (may be null): atomicMax of the number of sweeps taken.
// variant: 0 = one CTA up to l = 160, else the cluster; 1 = one CTA; 2 = cluster.
// C = alpha op(A) op(B) + beta C (op: 0 identity, 1 transpose; 32 x 32 tiles of C), and
// H = G ./ (s2_i^2 + s1_j^2) (or ./ (s2_i + s1_j) with squared) on the leading l x l.
cudaError_t launch_small_gemm(int M, int N, int K, float alpha, const float* A, int lda, int ta,
                              const float* B, int ldb, int tb, float beta, float* C, int ldc,
                              cudaStream_t st);
cudaError_t launch_round_bf16(float* x, int64_t rows, int cols, int64_t ld, cudaStream_t st);
cudaError_t launch_sylvester_scale(const float* G, int l, int lp, const float* s2, const float* s1,
                                   int squared, float* H, cudaStream_t st);

// SRFT test matrix (Section 4.6): the lc sampled frequencies (one CTA, at plan creation),
// then Omega n x cols_pad (2 lc real columns [Re, Im] per frequency, zero padding).
cudaError_t launch_srft_select(uint64_t seed, int64_t n, int lc, int* freq, cudaStream_t st);
cudaError_t launch_draw_srft(uint64_t seed, int64_t n, int lc, int cols_pad, const int* freq,
                             float* out, int64_t ld, __nv_bfloat16* out_t, int64_t ld_t,
                             cudaStream_t st);

// The modified SRFT (Section 4.6, eq. random_Givens): launch_gsrft_prepare writes, once
// per plan, the tables (gsrft_table_ints(n) ints): the permutations Pi, Pi' and the
// cos / sin of both rotation chains; launch_gsrft_apply turns the SRFT in omega (n x
// cols_pad, ld, columns >= ncols zero) into D'' Theta' D' Theta omega in place (scratch:
// n x ld floats).
cudaError_t launch_gsrft_prepare(uint64_t seed, int64_t n, int* tables, cudaStream_t st);
size_t gsrft_table_ints(int64_t n);
cudaError_t launch_gsrft_apply(uint64_t seed, int64_t n, int ncols, int cols_pad, const int* tables,
                               float* omega, float* scratch, int64_t ld, cudaStream_t st);

// The SRFT sketch as a transform along the rows of A (k_srft_fft.cu): y (m x ldy) gets
// [Re, Im] of l_c^-1/2 sum_j a_j d_j exp(-2 pi i j b_c / n) in columns 2c, 2c + 1 and zeros
// up to ldy.  adt: A float32 (0), bfloat16 (1), bfloat16 hi + lo (2, lo m rows further);
// n a power of two in [2048, 32768] (srft_fft_supported), lda even.  signs: n bits, bit j
// set where d_j = -1 (launch_srft_signs, from the SRFT draws of the seed).
bool srft_fft_supported(int64_t n);
cudaError_t launch_srft_signs(uint64_t seed, int64_t n, uint32_t* mask, cudaStream_t st);
cudaError_t launch_srft_fft(int adt, const void* A, int64_t lda, int64_t m, int64_t n,
                            const uint32_t* signs, const int* freq, int lc, float* y, int ldy,
                            int num_sms, cudaStream_t st);

// scratch: lp x lp floats of workspace (used by the cluster variant).
cudaError_t launch_jacobi_svd(const float* x, int64_t ldx, int transposed, int l, int lp,
                              float* ut, float* s, float* w, float* scratch, uint32_t* status,
                              uint32_t* info, cudaStream_t st, int variant = 0);
size_t jacobi_smem_bytes(int l);

// dst[r][c] = sum_{s < splits} src[s][r][c] for c < cols, 0 for cols <= c < cols_pad
// (layout change between the caller's leading dimension and the padded width).
cudaError_t launch_gather(const float* src, int splits, int64_t split_stride, int64_t lds,
                          float* dst, int64_t ldd, int64_t rows, int cols, int cols_pad,
                          cudaStream_t st);

// The same SVD on a thread-block cluster (block round-robin ordering), l <= 256.  With x_b,
// a second matrix of the same size and orientation (own outputs and scratch) runs in the
// same launch on a second cluster.
cudaError_t launch_jacobi_cluster(const float* x, int64_t ldx, int transposed, int l, int lp,
                                  float* ut, float* s, float* w, float* scratch, uint32_t* status,
                                  uint32_t* info, cudaStream_t st, const float* x_b = nullptr,
                                  float* ut_b = nullptr, float* s_b = nullptr, float* w_b = nullptr,
                                  float* scratch_b = nullptr);
// Two independent SVDs of the same size and orientation: one launch of the cluster kernel
// when it is the one launch_jacobi_svd would pick, else two launches.
cudaError_t launch_jacobi_svd_pair(const float* x, const float* x_b, int64_t ldx, int transposed, int l,
                                   int lp, float* ut, float* ut_b, float* s, float* s_b, float* w,
                                   float* w_b, float* scratch, float* scratch_b, uint32_t* status,
                                   uint32_t* info, cudaStream_t st, int variant);
cudaError_t prepare_jacobi_cluster();

// ---- backward (k_backward.cu) ----
// G = alpha A + beta G + L R^T (L: m x kr, ldl; R: n x kr, ldr; A float32 (adt 0),
// bfloat16 (1) or bfloat16 hi + lo (2, lo m * lda elements further); alpha = 0 skips A).
cudaError_t launch_lowrank_update(int64_t m, int64_t n, int kr, const float* L, int64_t ldl,
                                  const float* R, int64_t ldr, const void* A, int64_t lda, int adt,
                                  float alpha, float beta, float* G, int64_t ldg, cudaStream_t st);
// N = -copyltu(C) (lp x lp).
cudaError_t launch_copyltu_neg(const float* C, int lp, float* N, cudaStream_t st);
// M2 = M^T - K S^-1 of the SVD adjoint (see k_backward.cu).
cudaError_t launch_svd_adjoint(const float* J, const float* K, const float* s, const float* gS, int k,
                               int l, int lp, float* M2, cudaStream_t st);
// gUt = gU + rec (2 S^2 U - 2 S P) on the first k columns (rows x lp, zero beyond k).
cudaError_t launch_recon_cotangent(int64_t m, int k, int lp, const float* gU, const float* U,
                                   const float* P, const float* s, int rec, float* gUt, cudaStream_t st);
// Y (rows x lp) (+)= alpha X[:, :ncols] diag(c or 1/c), zero beyond ncols.
cudaError_t launch_colscale(int64_t rows, int ncols, int lp, const float* X, int lds, const float* c,
                            int inv, float alpha, int accumulate, float* Y, cudaStream_t st);
// out[j] = gS[j] + rec, j < k.
cudaError_t launch_gs_total(const float* gS, int k, int rec, float* out, cudaStream_t st);

// R^-1 of an upper triangular R (lp x lp, lp a multiple of 16 up to 256, the identity
// beyond l); block substitution, lp / 16 CTAs.
cudaError_t launch_trinv_upper(const float* r, int l, int lp, float* rinv, cudaStream_t st);

// Row ID (k_id.cu).  launch_id_pivot: Businger--Golub pivoting on the rows of res (m x lp,
// ld lp, overwritten by the residuals), l steps, one cooperative launch of `grid` CTAs
// (at most one per SM); coef (m x lp, zeroed by the caller) gets the coefficients of each
// row on the pivot directions, piv the l pivots in order (-1 from the step at which no
// row is left: ST_NUMERICAL); cand: id_cand_floats(grid, lp) floats; bar: one counter,
// zeroed by the caller.  launch_id_lt: Lt = C[J]^T (upper).  launch_gather_rows_t: out
// (n x lp) = A[J, :]^T for A float32 (0), bfloat16 (1), bfloat16 hi + lo (2).
cudaError_t launch_id_pivot(float* res, int64_t m, int l, int lp, float* coef, int* piv, float* cand,
                            unsigned* bar, uint32_t* status, int grid, cudaStream_t st);
size_t id_cand_floats(int grid, int lp);
cudaError_t launch_id_lt(const float* coef, const int* piv, int l, int lp, float* lt, cudaStream_t st);
cudaError_t launch_transpose_square(const float* src, int lp, float* dst, cudaStream_t st);
cudaError_t launch_gather_rows_t(int adt, const void* A, int64_t lda, int64_t m, int64_t n, const int* piv,
                                 int l, int lp, float* out, cudaStream_t st);

// Hermitian Stage B helpers: B <- (B + B^T) / 2 on the leading l x l (ld lp); eigenvalues
// from the SVD Ut S W^T of a symmetric matrix (mode 0: s_i sign(u_i . w_i)) or the squares
// s_i^2 (mode 1, the Nystrom factor's), k of them.
cudaError_t launch_symmetrize(float* B, int l, int lp, cudaStream_t st);
cudaError_t launch_eig_values(const float* ut, const float* w, const float* s, int l, int lp, int k,
                              int mode, float* out, cudaStream_t st);

// A bounded wait on `flag` (never set by the library) that records ST_TIMEOUT after `spins`
// polls and returns (rsvd_wait_selftest).
cudaError_t launch_wait_selftest(const uint32_t* flag, uint32_t spins, uint32_t* status,
                                 cudaStream_t st);

// One-time (per device) shared-memory attributes of the one-CTA kernels and of the
// tensor-core Gram and apply.
cudaError_t prepare_orth();
cudaError_t prepare_jacobi();
cudaError_t prepare_gram_tc();
cudaError_t prepare_apply_tc();

}  // namespace rsvd
