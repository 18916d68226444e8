// Gram matrix G = Y^T Y of a float32 sample on the tensor cores, the first step of a
// Cholesky-QR round (Algorithm 4.1 step 3 orthonormalises the sample; the rounds form
// G, factor G = R^T R and apply Q = Y R^-1).
//
// Precision: every float32 entry y is split exactly into three bfloat16 parts,
// y = h + m + t (h = bf16(y), m = bf16(y - h), t = y - h - m, each part carrying the
// next 8 bits of the significand), and
//   G ~= H^T H + H^T M + M^T H + H^T T + T^T H + M^T M,
// six BF16 products with float32 accumulation.  The products are exact and the terms
// left out (M^T T, T^T M, T^T T) are below 2^-24 of |Y|^T |Y| entrywise, but the tensor
// cores' float32 accumulation is not IEEE round-to-nearest: measured against a float64
// Gram, entries carry about 1e-6 of |Y|^T |Y| (a float32 FMA Gram over the same row blocks:
// about 1e-7), whatever the number of rows.  The bfloat16 tensor-core path, whose A is
// rounded to 2^-9, uses it; the plain float32 path keeps the FMA Gram.
//
// Layout: a stage holds 32 rows of Y (K = 32 of the MMAs) as three planes, each the
// MN-major, 128-byte-swizzled image of the rows' columns in 64-column boxes of 32 x 128
// bytes (column c of row k at box c / 64, byte k * 128 + (((c % 64) / 8) ^ (k % 8)) * 16
// + (c % 8) * 2).  Both MMA operands are these planes: A = columns 128 I .. 128 I + 127
// (the M side, tile I of the Gram's rows), B = columns 0 .. N_I - 1.  Tile 0 covers Gram
// rows 0..127 (N_0 = min(l_p, 128) columns, the lower triangle and the upper half of its
// diagonal block), tile 1 (l_p > 128) rows 128 .. l_p - 1 against all l_p columns.
//
// Work split: CTA b takes rows [b rows / G, (b + 1) rows / G) and writes its partial
// Gram matrix (lower triangle, row-major l_p x l_p) to gpart + b l_p^2; the reduce kernel
// sums the G partials in a fixed order.
//
// Warp roles (320 threads): warp 1 allocates tensor memory and issues the MMAs from one
// thread; warps 2..9 load Y (summing partial slabs, writing the sum out when asked),
// split it and store the planes, then drain the accumulators (warps 2..5 tile 0, 6..9
// tile 1; each warp reads the 32 tensor-memory lanes its index allows).  Every wait is
// bounded; on expiry the kernel records a timeout in the status word and winds down.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace rsvd {
namespace {

using namespace tcx;

constexpr int GKC = 32;                 // rows of Y per stage
constexpr int GBOX = GKC * 128;         // one 64-column box of one plane (bytes)
constexpr int GSTAGES = 4;
constexpr int GCONV = 8;                // loader/converter warps
constexpr int GTHREADS = 64 + 32 * GCONV;
constexpr int kPairs = 6;
__constant__ int c_pa[kPairs] = {0, 0, 1, 0, 2, 1};   // plane of A in product r
__constant__ int c_pb[kPairs] = {0, 1, 0, 2, 0, 1};   // plane of B in product r

// kind::f16 instruction descriptor with both operands MN-major: f32 accumulate, bf16 A
// and B, A and B transposed (bits 15, 16), N >> 3 in bits 17-22, M >> 4 in 24-28.
__host__ __device__ constexpr uint32_t idesc_mn_mn(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void split3(float v, float& h, float& m, float& t) {
  h = __bfloat162float(__float2bfloat16_rn(v));
  const float r = v - h;   // exact: the low 16 bits of v's significand
  m = __bfloat162float(__float2bfloat16_rn(r));
  t = r - m;               // exact, and a bfloat16 value (at most 8 significant bits)
}
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__global__ void __launch_bounds__(GTHREADS, 1)
    gram_tc_kernel(const float* __restrict__ src, int splits, int64_t split_stride,
                   float* __restrict__ y_out, int64_t rows, int lp, float* __restrict__ gpart,
                   uint32_t* status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar_full[GSTAGES], bar_empty[GSTAGES], bar_acc;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nt = lp > 128 ? 2 : 1;        // 128-row tiles of G
  const int nbox = 2 * nt;                // 64-column boxes per plane
  const uint32_t plane_bytes = (uint32_t)nbox * GBOX;
  const uint32_t stage_bytes = 3 * plane_bytes;
  const int n0 = lp < 128 ? lp : 128;     // columns of tile 0
  const int64_t r0 = (int64_t)blockIdx.x * rows / gridDim.x;
  const int64_t r1 = (int64_t)(blockIdx.x + 1) * rows / gridDim.x;
  const int nchunk = (int)((r1 - r0 + GKC - 1) / GKC) > 0 ? (int)((r1 - r0 + GKC - 1) / GKC) : 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < GSTAGES; ++s) {
      mbar_init(&bar_full[s], GCONV);
      mbar_init(&bar_empty[s], 1);
    }
    mbar_init(&bar_acc, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // Y is written by the launch before (which may still run); tensor memory is taken only
  // after it has finished, so this CTA never holds it while waiting.
  pdl_wait();
  pdl_trigger();
  const uint32_t tmem_cols = nt == 2 ? 512u : 128u;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  volatile int* abort_flag = &s_abort;

  if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t id0 = idesc_mn_mn(n0), id1 = idesc_mn_mn(lp);
      bool ok = true;
      for (int i = 0; i < nchunk; ++i) {
        const int s = i % GSTAGES;
        const uint32_t ph = (uint32_t)((i / GSTAGES) & 1);
        if (!mbar_wait(&bar_full[s], ph, abort_flag, status)) { ok = false; break; }
        tc_fence_after();
        const uint32_t base = smem_u32(smem + (size_t)s * stage_bytes);
#pragma unroll
        for (int j = 0; j < GKC / 16; ++j) {   // +16 rows of 128 bytes per k16 step
#pragma unroll
          for (int r = 0; r < kPairs; ++r) {
            const uint32_t pa = base + (uint32_t)c_pa[r] * plane_bytes + j * 2048;
            const uint32_t pb = base + (uint32_t)c_pb[r] * plane_bytes + j * 2048;
            const uint64_t bdesc = smem_desc(pb, GBOX, 1024);
            const uint32_t acc = (i | j | r) ? 1u : 0u;
            mma_bf16(tmem, smem_desc(pa, GBOX, 1024), bdesc, id0, acc);
            if (nt == 2) mma_bf16(tmem + 128, smem_desc(pa + 2 * GBOX, GBOX, 1024), bdesc, id1, acc);
          }
        }
        mma_commit(&bar_empty[s]);
      }
      if (ok) mma_commit(&bar_acc);
    }
  } else if (warp >= 2) {
    // ---------------- load, split, store; then drain ----------------
    const int ct = threadIdx.x - 64;            // 0 .. 32 GCONV - 1
    const int g4 = nbox * 16;                   // float4 groups per row of a stage
    const int per = GKC * g4 / (32 * GCONV);    // groups per thread: 4 or 8
    // the groups of chunk i this thread loads (all in flight at once); rows past this
    // CTA's range and columns past l_p read as zero
    auto load = [&](int i, float4 (&v)[8]) {
      const int64_t rb = r0 + (int64_t)i * GKC;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        const int g = ct + 32 * GCONV * u;
        const int k = g / g4, c = 4 * (g - k * g4);
        const int64_t row = rb + k;
        if (u < per && row < r1 && c < lp) {
          const int64_t off = row * lp + c;
          v[u] = *reinterpret_cast<const float4*>(src + off);
          for (int q = 1; q < splits; ++q) {
            const float4 w = *reinterpret_cast<const float4*>(src + off + (int64_t)q * split_stride);
            v[u].x += w.x; v[u].y += w.y; v[u].z += w.z; v[u].w += w.w;
          }
          if (y_out) *reinterpret_cast<float4*>(y_out + off) = v[u];
        }
      }
    };
    float4 cur[8], nxt[8];
    load(0, cur);
    for (int i = 0; i < nchunk; ++i) {
      if (i + 1 < nchunk) load(i + 1, nxt);
      const int s = i % GSTAGES;
      const uint32_t ph = (uint32_t)((i / GSTAGES) & 1);
      int ok = 1;
      if (lane == 0) ok = mbar_wait(&bar_empty[s], ph ^ 1u, abort_flag, status);
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      uint8_t* sp = smem + (size_t)s * stage_bytes;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (u >= per) break;
        const int g = ct + 32 * GCONV * u;
        const int k = g / g4, c = 4 * (g - k * g4);
        float h[4], m[4], t[4];
        split3(cur[u].x, h[0], m[0], t[0]);
        split3(cur[u].y, h[1], m[1], t[1]);
        split3(cur[u].z, h[2], m[2], t[2]);
        split3(cur[u].w, h[3], m[3], t[3]);
        const uint32_t o = (uint32_t)(c >> 6) * GBOX + (uint32_t)k * 128 +
                           ((uint32_t)(((c & 63) >> 3) ^ (k & 7)) << 4) + (uint32_t)(c & 7) * 2;
        *reinterpret_cast<uint2*>(sp + o) = make_uint2(pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]));
        *reinterpret_cast<uint2*>(sp + plane_bytes + o) =
            make_uint2(pack_bf16(m[0], m[1]), pack_bf16(m[2], m[3]));
        *reinterpret_cast<uint2*>(sp + 2 * plane_bytes + o) =
            make_uint2(pack_bf16(t[0], t[1]), pack_bf16(t[2], t[3]));
      }
      fence_proxy_async_smem();   // the planes are read by the tensor cores
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_full[s]);
#pragma unroll
      for (int u = 0; u < 8; ++u) cur[u] = nxt[u];
    }
    // drain: warp 2 + 4 I + q reads lanes 32 (warp % 4) .. + 31 of tile I
    const int tile = (warp - 2) >> 2, quad = warp & 3;
    if (tile < nt) {
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&bar_acc, 0, abort_flag, status));
      tc_fence_after();
      const int row = 128 * tile + 32 * quad + lane;
      const int ncols = tile == 0 ? n0 : lp;
      const uint32_t tb = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(128 * tile);
      float* gp = gpart + (int64_t)blockIdx.x * lp * lp + (int64_t)row * lp;
      for (int c0 = 0; c0 < ncols; c0 += 32) {
        float v[32];
        tmem_ld_cols(tb + c0, ncols - c0 >= 32 ? 32 : 16, v);
        if (!ok || row >= lp) continue;
#pragma unroll
        for (int e = 0; e < 32; ++e)
          if (c0 + e <= row && c0 + e < ncols) gp[c0 + e] = v[e];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols)
                 : "memory");
  }
}

size_t gram_tc_smem(int lp) {
  const int nt = lp > 128 ? 2 : 1;
  return (size_t)GSTAGES * 3 * (2 * nt) * GBOX + 1024;
}

}  // namespace

int gram_tc_grid(int64_t rows, int nblk_max) {
  int64_t g = cdiv(rows, (int64_t)GKC);
  if (g > kNumSMs) g = kNumSMs;
  if (g > nblk_max) g = nblk_max;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t prepare_gram_tc() {
  return cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)gram_tc_smem(256));
}

cudaError_t launch_gram_tc(const float* src, int splits, int64_t split_stride, float* y_out,
                           int64_t rows, int lp, float* gpart, int nblk, uint32_t* status,
                           cudaStream_t st) {
  if (lp < 16 || lp > 256 || lp % 16 != 0 || nblk < 1) return cudaErrorInvalidValue;
  return launch_pdl(gram_tc_kernel, dim3(nblk), dim3(GTHREADS), gram_tc_smem(lp), st, src, splits,
                    split_stride, y_out, rows, lp, gpart, status);
}

}  // namespace rsvd
