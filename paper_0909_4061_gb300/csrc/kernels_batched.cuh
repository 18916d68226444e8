// Launchers of the batched kernels (k_batched.cu): l <= 32, basis rows 32 float32
// wide, matrices concatenated by row offsets (roff: nb + 1 entries, device).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rsvd {

constexpr int kBatchedLP = 32;
constexpr int kBatchedStages = 8;

size_t batched_tc_smem(int stages, int fold);
cudaError_t prepare_batched();

// Grouped pass: units (matrix b, 128-row tile t) of Y_b = A_b X_b (mode 0) or
// Y_b = A_b^T X_b (mode 1); maps: nb tensor maps of A_b in device memory; map_x: host
// address of the operand's tensor map (passed by value; 64 rows hi + lo when fold = 1);
// kext/mext/xoff/yoff: per-matrix K extent, output rows, operand column offset, output
// row offset (device).
// grid: CTAs (units are dealt round-robin); stages: pipeline depth, 2 .. kBatchedStages
// (smem batched_tc_smem(stages, fold) per CTA; fewer stages let two CTAs share an SM).
cudaError_t launch_batched_tc(int mode, int fold, const void* maps, const void* map_x, const int2* units,
                              int nunits, const int64_t* kext, const int64_t* mext,
                              const int64_t* xoff, const int64_t* yoff, float* y, int grid,
                              uint32_t* status, cudaStream_t st, int stages = kBatchedStages);
cudaError_t launch_batched_draw(uint64_t seed, const int64_t* roff, int nb, int64_t total_rows, int l,
                                float* omega, __nv_bfloat16* xbf, int64_t ldx, const int64_t* xoff,
                                cudaStream_t st);
// Cholesky-QR rounds of every matrix's rows (matrix b from roff[b]) over 128-row units:
// units (b, tile) in matrix order, those of matrix b from ustart[b] (nb + 1 entries);
// part: nunits x 32 x 32 floats of Gram partials; rinv: nb x 32 x 32 scratch; rout gets
// the product of the rounds' R factors; shift_first: the first round factors G + s I,
// s = l u tr(G) (shifted Cholesky QR).  With xbf, the last round also writes Q as the next
// pass's operand (as launch_batched_to_bf16t does: matrix b at xbf + xoff[b], leading
// dimension ldx, with the lo half when split).  1 + 2 rounds launches.
cudaError_t launch_batched_cholqr(const float* yin, float* qout, const int64_t* roff, int nb, int l,
                                  int rounds, int shift_first, float* rout, float* rinv, const int2* units,
                                  int nunits, const int* ustart, float* part, uint32_t* status, cudaStream_t st,
                                  __nv_bfloat16* xbf = nullptr, int64_t ldx = 0, const int64_t* xoff = nullptr,
                                  int split = 0);
cudaError_t launch_batched_to_bf16t(const float* q, const int64_t* roff, int nb, int64_t total_rows,
                                    __nv_bfloat16* xbf, int64_t ldx, const int64_t* xoff, int split,
                                    cudaStream_t st);
cudaError_t launch_batched_jacobi(const float* x, int transposed, int l, int nb, float* ut, float* sig,
                                  float* w, uint32_t* status, uint32_t* info, cudaStream_t st);
// out rows of matrix b = its rows of q (nonzero in the first l columns) times the leading
// `valid` columns of its LP x LP small matrix (cols outputs per row); max_rows: the most
// rows any matrix has.
cudaError_t launch_batched_lift(const float* q, const int64_t* roff, int nb, int64_t max_rows, int l,
                                const float* small, int cols, int valid, float* out, int ldo,
                                cudaStream_t st);

// ---- backward (k_batched_bwd.cu) ----
// gQ = (P (I - 2 S) + 2 U S^2) Ut_k^T with U = Q Ut_k (per row; P = A V, m side), and
// ublk = U (I - 2 S) (first k columns, zero beyond), ld ldu.
// (l: the basis width, columns of Q beyond it are zero; k <= l; ldu a multiple of 4 and
// ublk 16-byte aligned)
cudaError_t launch_bwd_gq(const float* P, const float* Q, const int64_t* roff, const int2* units, int nunits,
                          int l, const float* ut, const float* sig, int k, float* gq, float* ublk, int ldu,
                          cudaStream_t st);
// per matrix: N = copyltu(-gQ^T Q) (from partials over the Cholesky-QR units: units /
// nunits / ustart, part: nunits x 32 x 32) and Rinv = R^-1 (R upper, l x l, identity beyond l)
cudaError_t launch_bwd_qr_small(const float* Q, const float* gQ, const int64_t* roff, const int2* units,
                                int nunits, const int* ustart, int nb, int l, const float* R, float* part,
                                float* N, float* Rinv, cudaStream_t st);
// gY = (gQ + Q N) R^-T, per row (over the Cholesky-QR units of the side)
cudaError_t launch_bwd_qr_apply(const float* Q, const float* gQ, const int64_t* roff, const int2* units,
                                int nunits, int l, const float* N, const float* Rinv, float* gY, cudaStream_t st);
// dst[r][col0 + c] = src[r][c] (rows x 32 -> ld ldd)
cudaError_t launch_copy_block(const float* src, int64_t rows, float* dst, int ldd, int col0,
                              cudaStream_t st);
// planes [3][n] = the three-way bfloat16 split of x (n floats): h, m, t with
// x = h + m + t to 24 significant bits.
cudaError_t launch_bwd_split(const float* x, int64_t n, __nv_bfloat16* planes, cudaStream_t st);
cudaError_t prepare_batched_bwd();
int bwd_final_tile();   // rows and columns of a unit of launch_bwd_final
// gA_b = 2 A_b + L_b R_b^T on the tensor cores over units (b, row tile, column tile) of
// bwd_final_tile() x bwd_final_tile(); map_l / map_r: host addresses of the tensor maps of
// the split planes of L (3 sum_m rows of kr bf16) and R (3 sum_n rows), box 64 x 128;
// maps_a: device array of the per-matrix tensor maps of A_b (box 64 columns x 128 rows);
// kr a multiple of 64; grid: persistent CTAs (one per SM).
cudaError_t launch_bwd_final(const void* map_l, const void* map_r, const void* maps_a, const int4* units,
                             int nunits, int64_t sum_m, int64_t sum_n, int kr, float* const* gA,
                             const int64_t* m, const int64_t* n, const int64_t* roff_m, const int64_t* roff_n,
                             int grid, uint32_t* status, cudaStream_t st);

}  // namespace rsvd
