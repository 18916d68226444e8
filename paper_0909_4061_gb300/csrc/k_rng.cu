// Draw of the Gaussian test matrix Omega (Algorithm 4.1 step 1; Algorithm 4.4
// step 1) from the counter-based generator of philox.cuh.  One thread per
// (row i, column group g): four normals for columns 4g .. 4g+3.
#include "common.cuh"
#include "kernels.cuh"
#include "philox.cuh"

namespace rsvd {
namespace {

__global__ void draw_gaussian_kernel(uint2 key, uint32_t stream_id, int64_t rows, int cols,
                                     int cols_pad, float* __restrict__ out, int64_t ld,
                                     __nv_bfloat16* __restrict__ out_t, int64_t ld_t) {
  const int groups = (cols_pad + 3) / 4;
  const int64_t n = rows * groups;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows;  // consecutive threads take consecutive rows
    const int g = (int)(e / rows);
    float z[4] = {0.f, 0.f, 0.f, 0.f};
    if (4 * g < cols) {
      const float4 v = gaussian4(key, (uint32_t)g, (uint32_t)i, stream_id);
      z[0] = v.x; z[1] = v.y; z[2] = v.z; z[3] = v.w;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int j = 4 * g + t;
      if (j >= cols_pad) break;
      const float val = (j < cols) ? z[t] : 0.0f;
      if (out) out[i * ld + j] = val;
      if (out_t) out_t[(int64_t)j * ld_t + i] = __float2bfloat16_rn(val);
    }
  }
}

}  // namespace

cudaError_t launch_draw_gaussian(uint64_t seed, uint32_t stream_id, int64_t rows, int cols,
                                 int cols_pad, float* out, int64_t ld, __nv_bfloat16* out_t,
                                 int64_t ld_t, cudaStream_t st) {
  if (rows <= 0 || cols_pad <= 0) return cudaSuccess;
  if (cols_pad < cols) return cudaErrorInvalidValue;
  const int64_t n = rows * ((cols_pad + 3) / 4);
  const int64_t blocks = cdiv(n, 256);
  const unsigned grid = (unsigned)(blocks < 16 * kNumSMs ? blocks : 16 * kNumSMs);
  draw_gaussian_kernel<<<grid, 256, 0, st>>>(seed_key(seed), stream_id, rows, cols, cols_pad, out,
                                             ld, out_t, ld_t);
  return cudaGetLastError();
}

}  // namespace rsvd
