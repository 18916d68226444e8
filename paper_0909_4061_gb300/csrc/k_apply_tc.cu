// Q = Y R^-1 on the tensor cores for wide bases (the apply step of a Cholesky-QR round,
// Algorithm 4.1 step 3's orthonormalisation), Y float32 (rows x l_p), R^-1 upper
// triangular (l_p x l_p, zero padded), Q float32.
//
// Precision: Y and R^-1 are split exactly into three bfloat16 parts each (y = h + m + t,
// as for the tensor-core Gram) and Q ~= H Rh + H Rm + M Rh + H Rt + T Rh + M Rm, six
// products with float32 accumulation in tensor memory.  As for the Gram, the
// accumulation is not IEEE-exact (about 1e-6 relative), which the bfloat16 path, whose A
// is rounded to 2^-9, absorbs.
//
// Layout: a stage covers 32 columns of Y (K = 32).  The A side (128 rows of Y) is three
// K-major planes with 64-byte rows and the 64-byte swizzle (16-byte chunk c of row m at
// chunk c ^ ((m / 2) % 4)), written by the loader warps from registers.  The B side is
// rows 32 kc .. 32 kc + 31 of R^-1's planes, MN-major with the 128-byte swizzle in boxes
// of 64 columns x 32 rows, copied from an image that apply_tc_prep writes once per round.
// R^-1 is upper triangular, so chunk kc only meets columns n >= 32 kc: its MMAs start at
// box kc / 2 and are l_p - 64 (kc / 2) wide.
//
// Work split: 128-row tiles, tile t by CTA t mod G (persistent); two accumulators of l_p
// columns (32-column aligned) let the MMAs of a tile run while the previous tile is
// written out.
//
// Warp roles (320 threads): warp 0 copies the B image chunks (bulk copies), warp 1 owns
// tensor memory and issues the MMAs from one thread, warps 2..5 load, split and store
// the A chunks, warps 6..9 drain the accumulators to Q.  Every wait is bounded; on expiry
// the kernel records a timeout in the status word and winds down.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace rsvd {
namespace {

using namespace tcx;

constexpr int AKC = 32;                   // columns of Y (K) per stage
constexpr int ABOX = AKC * 128;           // one 64-column box of one B plane (bytes)
constexpr int AAPL = BM * AKC * 2;        // one A plane of a stage (bytes): 8 KB
constexpr int ASTAGES = 3;
constexpr int ATHREADS = 320;
constexpr int kPairs = 6;
__constant__ int c_qa[kPairs] = {0, 0, 1, 0, 2, 1};   // plane of Y in product r
__constant__ int c_qb[kPairs] = {0, 1, 0, 2, 0, 1};   // plane of R^-1 in product r

// kind::f16, f32 accumulate, bf16 A (K-major) and B (MN-major: bit 16), N >> 3 in bits
// 17-22, M >> 4 in 24-28
__host__ __device__ constexpr uint32_t idesc_k_mn(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void split3(float v, float& h, float& m, float& t) {
  h = __bfloat162float(__float2bfloat16_rn(v));
  const float r = v - h;
  m = __bfloat162float(__float2bfloat16_rn(r));
  t = r - m;
}
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// R^-1 image: chunk kc, plane p, box b at ((kc * 3 + p) * nbox + b) * ABOX bytes; in a box,
// row r (k = 32 kc + r) and column n (b * 64 + c) at r * 128 + ((c / 8) ^ (r % 8)) * 16 +
// (c % 8) * 2.  Entries past l_p (rows or columns) are zero.
__global__ void apply_tc_prep_kernel(const float* __restrict__ rinv, int lp, int nbox,
                                     uint8_t* __restrict__ img) {
  pdl_wait();
  pdl_trigger();
  const int nkc = (lp + AKC - 1) / AKC;
  const int ncol = nbox * 64;
  const int total = nkc * AKC * ncol;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int n = e % ncol, k = e / ncol;
    const int kc = k / AKC, r = k % AKC, b = n >> 6, c = n & 63;
    const float v = (k < lp && n < lp) ? rinv[(int64_t)k * lp + n] : 0.0f;
    float h, m, t;
    split3(v, h, m, t);
    const uint32_t off = (uint32_t)r * 128 + ((uint32_t)((c >> 3) ^ (r & 7)) << 4) + (uint32_t)(c & 7) * 2;
    const float parts[3] = {h, m, t};
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      uint8_t* dst = img + ((size_t)(kc * 3 + p) * nbox + b) * ABOX + off;
      *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(parts[p]);
    }
  }
}

__global__ void __launch_bounds__(ATHREADS, 1)
    apply_tc_kernel(const float* __restrict__ y, float* __restrict__ q, int64_t rows, int lp,
                    const uint8_t* __restrict__ img, uint32_t* status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar_full[ASTAGES], bar_empty[ASTAGES], bar_af[2], bar_ae[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nbox = (lp + 63) / 64;
  const int nkc = (lp + AKC - 1) / AKC;
  const uint32_t bplane = (uint32_t)nbox * ABOX;
  const uint32_t stage_bytes = 3 * AAPL + 3 * bplane;    // A planes, then B planes
  const int64_t ntile = (rows + BM - 1) / BM;

  if (threadIdx.x == 0) {
    for (int s = 0; s < ASTAGES; ++s) {
      mbar_init(&bar_full[s], 4 + 1);   // the four loader warps and the copy's transaction
      mbar_init(&bar_empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&bar_af[a], 1);
      mbar_init(&bar_ae[a], 4);
    }
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // Y and the image come from the launches before; tensor memory is taken only after
  // they have finished, so this CTA never holds it while waiting.
  pdl_wait();
  pdl_trigger();
  const uint32_t acc_stride = (uint32_t)((lp + 31) & ~31);   // the two accumulators
  uint32_t tmem_cols = 32;
  while (tmem_cols < 2u * acc_stride) tmem_cols <<= 1;
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

  if (warp == 0) {
    // ---------------- B image chunks ----------------
    if (lane == 0) {
      int64_t i = 0;
      for (int64_t t = blockIdx.x; t < ntile; t += gridDim.x) {
        for (int kc = 0; kc < nkc; ++kc, ++i) {
          const int s = (int)(i % ASTAGES);
          const uint32_t ph = (uint32_t)((i / ASTAGES) & 1);
          if (!mbar_wait(&bar_empty[s], ph ^ 1u, abort_flag, status)) { t = ntile; break; }
          const int b0 = kc >> 1;
          const uint32_t run = (uint32_t)(nbox - b0) * ABOX;
          uint8_t* sb = smem + (size_t)s * stage_bytes + 3 * AAPL;
          mbar_expect_tx(&bar_full[s], 3 * run);
#pragma unroll
          for (int p = 0; p < 3; ++p)
            bulk_copy(sb + p * bplane, img + ((size_t)(kc * 3 + p) * nbox + b0) * ABOX, run, &bar_full[s]);
        }
      }
      // let the copies still in flight land before the CTA can exit
      for (int64_t j = (i > ASTAGES ? i - ASTAGES : 0); j < i; ++j) {
        const int s = (int)(j % ASTAGES);
        const uint32_t ph = (uint32_t)((j / ASTAGES) & 1);
        for (uint32_t w = 0; w < kSpinLimit && !mbar_try_wait(&bar_full[s], ph); ++w) __nanosleep(64);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int64_t i = 0;
      int tl = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntile && ok; t += gridDim.x, ++tl) {
        const int ab = tl & 1;
        const uint32_t acc = tmem + (uint32_t)ab * acc_stride;
        if (!mbar_wait(&bar_ae[ab], ((uint32_t)(tl >> 1) & 1u) ^ 1u, abort_flag, status)) break;
        tc_fence_after();
        for (int kc = 0; kc < nkc; ++kc, ++i) {
          const int s = (int)(i % ASTAGES);
          const uint32_t ph = (uint32_t)((i / ASTAGES) & 1);
          if (!mbar_wait(&bar_full[s], ph, abort_flag, status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + (size_t)s * stage_bytes);
          const uint32_t sb = sa + 3 * AAPL;
          const int b0 = kc >> 1;
          const uint32_t id = idesc_k_mn(lp - 64 * b0);
#pragma unroll
          for (int j = 0; j < AKC / 16; ++j) {
#pragma unroll
            for (int r = 0; r < kPairs; ++r) {
              // A: K-major, 64-byte swizzle, 8-row groups 512 B apart, +32 B per k16 step;
              // B: MN-major, 128-byte swizzle, boxes ABOX apart, +16 rows of 128 B per step
              const uint64_t adesc = smem_desc(sa + (uint32_t)c_qa[r] * AAPL + j * 32, 16, 512, 4);
              const uint64_t bdesc = smem_desc(sb + (uint32_t)c_qb[r] * bplane + j * 2048, ABOX, 1024);
              mma_bf16(acc + 64 * b0, adesc, bdesc, id, (kc | j | r) ? 1u : 0u);
            }
          }
          mma_commit(&bar_empty[s]);
        }
        if (ok) mma_commit(&bar_af[ab]);
      }
    }
  } else if (warp < 6) {
    // ---------------- load, split, store the A chunks ----------------
    const int ct = threadIdx.x - 64;   // 0..127
    // chunk: 128 rows x 32 columns = 1024 float4 groups, 8 per thread (row g / 8, cols 4 (g % 8))
    auto load = [&](int64_t t, int kc, float4 (&v)[8]) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int g = ct + 128 * u;
        const int m = g >> 3, c = kc * AKC + 4 * (g & 7);
        const int64_t row = t * BM + m;
        v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < rows && c < lp) v[u] = *reinterpret_cast<const float4*>(y + row * lp + c);
      }
    };
    float4 cur[8], nxt[8];
    int64_t t = blockIdx.x;
    int kc = 0;
    if (t < ntile) load(t, 0, cur);
    for (int64_t i = 0; t < ntile; ++i) {
      int64_t tn = t;
      int kn = kc + 1;
      if (kn == nkc) { kn = 0; tn += gridDim.x; }
      if (tn < ntile) load(tn, kn, nxt);
      const int s = (int)(i % ASTAGES);
      const uint32_t ph = (uint32_t)((i / ASTAGES) & 1);
      int ok = 1;
      if (lane == 0) ok = mbar_wait(&bar_empty[s], ph ^ 1u, abort_flag, status);
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      uint8_t* sa = smem + (size_t)s * stage_bytes;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int g = ct + 128 * u;
        const int m = g >> 3, kk = 4 * (g & 7);
        float h[4], mm[4], tt[4];
        split3(cur[u].x, h[0], mm[0], tt[0]);
        split3(cur[u].y, h[1], mm[1], tt[1]);
        split3(cur[u].z, h[2], mm[2], tt[2]);
        split3(cur[u].w, h[3], mm[3], tt[3]);
        const uint32_t o = (uint32_t)m * 64 + ((uint32_t)((kk >> 3) ^ ((m >> 1) & 3)) << 4) + (uint32_t)(kk & 7) * 2;
        *reinterpret_cast<uint2*>(sa + o) = make_uint2(pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]));
        *reinterpret_cast<uint2*>(sa + AAPL + o) = make_uint2(pack_bf16(mm[0], mm[1]), pack_bf16(mm[2], mm[3]));
        *reinterpret_cast<uint2*>(sa + 2 * AAPL + o) = make_uint2(pack_bf16(tt[0], tt[1]), pack_bf16(tt[2], tt[3]));
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_full[s]);
#pragma unroll
      for (int u = 0; u < 8; ++u) cur[u] = nxt[u];
      t = tn;
      kc = kn;
    }
  } else {
    // ---------------- drain: warps 6..9, lanes 32 (warp % 4) .. + 31 ----------------
    const int quad = warp & 3;
    int tl = 0;
    for (int64_t t = blockIdx.x; t < ntile; t += gridDim.x, ++tl) {
      const int ab = tl & 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&bar_af[ab], (uint32_t)(tl >> 1) & 1u, abort_flag, status));
      tc_fence_after();
      const int64_t row = t * BM + 32 * quad + lane;
      const uint32_t tb = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)ab * acc_stride;
      for (int c0 = 0; c0 < lp; c0 += 32) {
        float v[32];
        tmem_ld_cols(tb + c0, lp - c0 >= 32 ? 32 : 16, v);
        if (!ok || row >= rows) continue;
        float* dst = q + row * lp + c0;
#pragma unroll
        for (int e = 0; e < 32; e += 4)
          if (c0 + e < lp) *reinterpret_cast<float4*>(dst + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_ae[ab]);
      if (!ok) break;
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

size_t apply_tc_smem(int lp) {
  const int nbox = (lp + 63) / 64;
  return (size_t)ASTAGES * (3 * AAPL + 3 * (size_t)nbox * ABOX) + 1024;
}

}  // namespace

size_t apply_tc_image_bytes(int lp) {
  const int nbox = (lp + 63) / 64, nkc = (lp + AKC - 1) / AKC;
  return (size_t)nkc * 3 * nbox * ABOX;
}

cudaError_t prepare_apply_tc() {
  return cudaFuncSetAttribute(apply_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)apply_tc_smem(256));
}

cudaError_t launch_apply_tc(const float* y, float* q, int64_t rows, int lp, const float* rinv,
                            void* img, uint32_t* status, cudaStream_t st) {
  if (lp < 16 || lp > 256 || lp % 16 != 0 || rows < 1) return cudaErrorInvalidValue;
  const int nbox = (lp + 63) / 64;
  cudaError_t e = launch_pdl(apply_tc_prep_kernel, dim3(64), dim3(256), 0, st, rinv, lp, nbox,
                             static_cast<uint8_t*>(img));
  if (e != cudaSuccess) return e;
  const int64_t ntile = cdiv(rows, (int64_t)BM);
  const int grid = (int)(ntile < kNumSMs ? ntile : kNumSMs);
  return launch_pdl(apply_tc_kernel, dim3(grid), dim3(ATHREADS), apply_tc_smem(lp), st, y, q, rows,
                    lp, static_cast<const uint8_t*>(img), status);
}

}  // namespace rsvd
