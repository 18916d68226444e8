// Shared device/host helpers of the GB300 randomized SVD library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/rsvd.h"

namespace rsvd {

// ---- device status word bits (plan->status) --------------------------------
enum : uint32_t {
  ST_NONFINITE = 1u,        // NaN/Inf in a Gram diagonal or a pivot
  ST_NUMERICAL = 2u,        // breakdown the safeguards could not absorb
  ST_RANK_DEFICIENT = 4u,   // a Cholesky pivot was replaced (informational)
  ST_TIMEOUT = 8u,          // a bounded wait expired
  ST_JACOBI_NOCONV = 16u,   // Jacobi hit its sweep limit (informational)
};

constexpr int kNumSMs = 152;          // GB300: 2 dies x 76 SMs (queried at run time too)
constexpr int kMaxL = 256;            // largest basis width l = k + p supported
constexpr float kEpsF32 = 5.9604645e-08f;  // 2^-24, unit roundoff of float32

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline int64_t round_up(int64_t a, int64_t b) { return cdiv(a, b) * b; }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void set_status(uint32_t* status, uint32_t bit) {
  if (status) atomicOr(status, bit);
}

// Programmatic dependent launch.  A kernel launched with launch_pdl may start before its
// predecessor in the stream has finished; pdl_wait() blocks until that predecessor has
// completed and its writes are visible.  Every kernel that lets its dependents start
// early (pdl_trigger) does so only after its own pdl_wait(), so when a kernel starts,
// every kernel two or more launches back has completed: code before pdl_wait() may read
// their outputs, and nothing else.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace rsvd

#define RSVD_CUDA_TRY(expr)                          \
  do {                                               \
    cudaError_t _e = (expr);                         \
    if (_e != cudaSuccess) return RSVD_ERR_CUDA;     \
  } while (0)
