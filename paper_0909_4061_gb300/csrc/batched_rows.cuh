// Row tiles of the batched path in shared memory.  A Cholesky-QR unit is 128 consecutive
// rows of one matrix's tall factor (32 floats a row, zero beyond the basis width l).  The
// kernels that work a thread per row stage the unit with coalesced 16-byte loads into rows
// of kRowStride = 36 floats: a quarter-warp's 16-byte stores then fill one row (32 banks),
// and a thread's 16-byte reads of its own row, 36 floats from its neighbour's, fall in
// distinct banks too.  Results leave the same way, by coalesced 16-byte stores.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rsvd {

constexpr int kTileRows = 128;     // rows of a unit = threads of a row kernel
constexpr int kTileWidth = 32;     // floats of a row in global memory
constexpr int kRowStride = 36;     // floats of a staged row

// rows row0 .. row0 + nr - 1 of src (row length kTileWidth) into ys; column blocks
// c4 >= L4 (4 columns each) and rows >= nr read as zero.  Every thread's loads are issued
// before its first store.  kTileRows threads.
template <int L4>
__device__ __forceinline__ void stage_tile(const float* __restrict__ src, int64_t row0, int nr, float* ys) {
  constexpr int N = kTileRows * (kTileWidth / 4) / kTileRows;   // 8 float4 per thread
  const int c4 = threadIdx.x & 7;                                // the same column block every step
  float4 v[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int rr = (threadIdx.x + k * kTileRows) >> 3;
    v[k] = (rr < nr && c4 < L4) ? reinterpret_cast<const float4*>(src + (row0 + rr) * kTileWidth)[c4]
                                : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int rr = (threadIdx.x + k * kTileRows) >> 3;
    *reinterpret_cast<float4*>(ys + rr * kRowStride + 4 * c4) = v[k];
  }
}

// rows 0 .. nr - 1 of ys to dst + (row0 + r) * ld (ld a multiple of 4, dst 16-byte
// aligned), all kTileWidth columns, zeros for column blocks c4 >= L4.  kTileRows threads.
template <int L4>
__device__ __forceinline__ void store_tile(const float* ys, int nr, float* __restrict__ dst, int64_t row0,
                                           int64_t ld) {
  const int c4 = threadIdx.x & 7;
#pragma unroll
  for (int k = 0; k < kTileRows * (kTileWidth / 4) / kTileRows; ++k) {
    const int rr = (threadIdx.x + k * kTileRows) >> 3;
    if (rr < nr)
      *reinterpret_cast<float4*>(dst + (row0 + rr) * ld + 4 * c4) =
          c4 < L4 ? *reinterpret_cast<const float4*>(ys + rr * kRowStride + 4 * c4) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// 16-byte global -> shared copy through L2 (cp.async.cg) that lands without passing through
// registers, zero-filled (no global read) when !valid
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most N of this thread's committed groups are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// stage_tile by cp.async: the copies are issued and left in flight (commit and wait are
// the caller's); column blocks c4 >= L4 are not copied (a caller that reads them must not)
template <int L4>
__device__ __forceinline__ void stage_tile_async(const float* __restrict__ src, int64_t row0, int nr, float* ys) {
  const int c4 = threadIdx.x & 7;
  if (c4 >= L4) return;
#pragma unroll
  for (int k = 0; k < kTileRows * (kTileWidth / 4) / kTileRows; ++k) {
    const int rr = (threadIdx.x + k * kTileRows) >> 3;
    const bool valid = rr < nr;
    cp_async16(ys + rr * kRowStride + 4 * c4, src + (row0 + (valid ? rr : 0)) * kTileWidth + 4 * c4, valid);
  }
}

// the first 4 L4 floats of row t of ys into registers
template <int L4>
__device__ __forceinline__ void load_row(const float* ys, int t, float (&y)[4 * L4]) {
#pragma unroll
  for (int c4 = 0; c4 < L4; ++c4) {
    const float4 v = *reinterpret_cast<const float4*>(ys + t * kRowStride + 4 * c4);
    y[4 * c4] = v.x; y[4 * c4 + 1] = v.y; y[4 * c4 + 2] = v.z; y[4 * c4 + 3] = v.w;
  }
}

}  // namespace rsvd
