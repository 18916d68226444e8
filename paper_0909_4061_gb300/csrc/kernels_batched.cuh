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
cudaError_t launch_batched_tc(int mode, int fold, const void* maps, const void* map_x, const int2* units,
                              int nunits, const int64_t* kext, const int64_t* mext,
                              const int64_t* xoff, const int64_t* yoff, float* y, int grid,
                              uint32_t* status, cudaStream_t st);
cudaError_t launch_batched_draw(uint64_t seed, const int64_t* roff, int nb, int64_t total_rows, int l,
                                float* omega, __nv_bfloat16* xbf, int64_t ldx, const int64_t* xoff,
                                cudaStream_t st);
cudaError_t launch_batched_cholqr(const float* yin, float* qout, const int64_t* roff, int nb, int l,
                                  int rounds, float* rout, uint32_t* status, cudaStream_t st);
cudaError_t launch_batched_to_bf16t(const float* q, const int64_t* roff, int nb, int64_t total_rows,
                                    __nv_bfloat16* xbf, int64_t ldx, const int64_t* xoff, int split,
                                    cudaStream_t st);
cudaError_t launch_batched_jacobi(const float* x, int transposed, int l, int nb, float* ut, float* sig,
                                  float* w, uint32_t* status, uint32_t* info, cudaStream_t st);
cudaError_t launch_batched_lift(const float* q, const int64_t* roff, int nb, int64_t total_rows,
                                const float* small, int cols, float* out, int ldo, cudaStream_t st);

}  // namespace rsvd
