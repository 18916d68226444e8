// Batched randomized SVD of many small matrices (l <= 32): every step of
// Algorithm 4.4 + Algorithm 5.1 as one launch over the whole batch.
//
// Layout: the matrices' row blocks are concatenated (matrix b's m_b rows start at
// row roff[b] of an m-side buffer, its n_b rows at a separate offset on the n side),
// every row LP = 32 float32 wide; the transposed bfloat16 operand of a pass is
// one LP x sum(K) array with matrix b's columns from xoff[b] (a multiple of 8:
// 16-byte aligned TMA coordinates).  Per-matrix small matrices (R factors, the
// l x l SVD) are LP x LP blocks at b * LP * LP.
//
// Kernels:
//   batched_tc_kernel<MODE> : grouped tensor-core pass; a unit is one 128-row tile of
//                             one matrix with all its k tiles; CTAs take units
//                             round-robin; A_b through per-matrix tensor maps in global
//                             memory, the operand through one map; double-buffered
//                             accumulator in tensor memory.
//   batched_draw_kernel     : Omega_b from seed + b (Philox, stream 0), rounded to
//                             bfloat16: the transposed operand and its float32 copy.
//   bqr_*_kernel            : Cholesky-QR rounds over 128-row units of all matrices
//                             (Gram partials, one CTA per matrix for the 32 x 32 factor,
//                             its inverse and the product of the R factors, a thread per
//                             row for the apply, whose last round also writes the next
//                             pass's operand).
//   batched_to_bf16t_kernel : basis -> transposed bfloat16 operand (the backward's).
//   batched_jacobi_kernel   : one CTA per matrix: one-sided Jacobi of an l x l matrix,
//                             a half-warp per column pair, sorted outputs.
//   batched_lift_kernel     : rows of Q_b times the leading columns of a small matrix,
//                             a thread per row.
#include <cuda.h>

#include "common.cuh"
#include "batched_rows.cuh"
#include "kernels_batched.cuh"
#include "philox.cuh"
#include "tc_ptx.cuh"

namespace rsvd {
namespace {

using namespace tcx;

constexpr int LPB = 32;              // padded basis width of the batched path
constexpr int kBThreads = 192;

__device__ __forceinline__ int find_matrix(const int64_t* __restrict__ off, int nb, int64_t r) {
  int lo = 0, hi = nb - 1;   // largest b with off[b] <= r
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// grouped tensor-core pass
// ---------------------------------------------------------------------------
// FOLD: the operand carries a bfloat16 hi part (rows 0..31) and the residual lo part
// (rows 32..63) of a float32 basis; one MMA with N = 64 and the epilogue adds the two
// halves, so the pass sees the basis to about 16 significant bits.
template <int MODE, int FOLD>
__global__ void __launch_bounds__(kBThreads, 1) batched_tc_kernel(
    const CUtensorMap* __restrict__ maps, const __grid_constant__ CUtensorMap map_x,
    const int2* __restrict__ units, int nunits, const int64_t* __restrict__ kext,
    const int64_t* __restrict__ mext, const int64_t* __restrict__ xoff,
    const int64_t* __restrict__ yoff, float* __restrict__ y, int stages, uint32_t* status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar_full[16], bar_empty[16], bar_acc_full[2], bar_acc_empty[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  constexpr uint32_t a_bytes = BM * BK * 2;
  constexpr int NX = LPB * (FOLD ? 2 : 1);   // operand rows = MMA N
  constexpr uint32_t x_bytes = NX * BK * 2;
  constexpr uint32_t stage_bytes = a_bytes + x_bytes;
  constexpr uint32_t acc_cols = NX;
  constexpr uint32_t tmem_cols = 2 * acc_cols;

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&bar_full[s], 1);
      mbar_init(&bar_empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&bar_acc_full[a], 1);
      mbar_init(&bar_acc_empty[a], 4);
    }
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
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
    if (lane == 0) {
      int64_t i = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        const int b = units[u].x, t = units[u].y;
        const CUtensorMap* ma = maps + b;
        // the maps were written through the generic proxy (a copy before the launch)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                         reinterpret_cast<uint64_t>(ma))
                     : "memory");
        const int kt = (int)cdiv(kext[b], BK);
        const int xo = (int)xoff[b];
        for (int kk = 0; kk < kt; ++kk, ++i) {
          const int s = (int)(i % stages);
          const uint32_t ph = (uint32_t)((i / stages) & 1);
          if (!mbar_wait(&bar_empty[s], ph ^ 1u, abort_flag, status)) { ok = false; break; }
          uint8_t* sa = smem + (size_t)s * stage_bytes;
          uint8_t* sx = sa + a_bytes;
          mbar_expect_tx(&bar_full[s], stage_bytes);
          if (MODE == 0) {
            tma_load_2d(sa, ma, &bar_full[s], kk * BK, t * BM);
          } else {
            tma_load_2d(sa, ma, &bar_full[s], t * BM, kk * BK);
            tma_load_2d(sa + 8192, ma, &bar_full[s], t * BM + 64, kk * BK);
          }
          tma_load_2d(sx, &map_x, &bar_full[s], xo + kk * BK, 0);
        }
      }
      const int64_t issued = i;
      for (int64_t j = (issued > stages ? issued - stages : 0); j < issued; ++j) {
        const int s = (int)(j % stages);
        const uint32_t ph = (uint32_t)((j / stages) & 1);
        for (uint32_t w = 0; w < kSpinLimit && !mbar_try_wait(&bar_full[s], ph); ++w) __nanosleep(64);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = instr_desc(NX, MODE);
      int64_t i = 0;
      int j = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x, ++j) {
        const int b = units[u].x;
        const int kt = (int)cdiv(kext[b], BK);
        const int ab = j & 1;
        if (!mbar_wait(&bar_acc_empty[ab], ((uint32_t)(j >> 1) & 1u) ^ 1u, abort_flag, status)) break;
        tc_fence_after();
        const uint32_t dst = tmem + ab * acc_cols;
        for (int kk = 0; kk < kt; ++kk, ++i) {
          const int s = (int)(i % stages);
          const uint32_t ph = (uint32_t)((i / stages) & 1);
          if (!mbar_wait(&bar_full[s], ph, abort_flag, status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + (size_t)s * stage_bytes);
          const uint32_t sx = sa + a_bytes;
#pragma unroll
          for (int q = 0; q < BK / 16; ++q) {
            const uint64_t adesc = MODE == 0 ? smem_desc(sa + q * 32, 16, 1024)
                                             : smem_desc(sa + q * 2048, 8192, 1024);
            const uint64_t bdesc = smem_desc(sx + q * 32, 16, 1024);
            mma_bf16(dst, adesc, bdesc, idesc, (kk == 0 && q == 0) ? 0u : 1u);
          }
          mma_commit(&bar_empty[s]);
        }
        if (ok) mma_commit(&bar_acc_full[ab]);
      }
    }
  } else {
    const int quad = warp & 3;
    const int row = quad * 32 + lane;
    int j = 0;
    for (int u = blockIdx.x; u < nunits; u += gridDim.x, ++j) {
      const int b = units[u].x, t = units[u].y;
      const int ab = j & 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&bar_acc_full[ab], (uint32_t)(j >> 1) & 1u,
                                                        abort_flag, status));
      tc_fence_after();
      if (ok) {
        float v[32];
        tmem_ld32(tmem + ab * acc_cols + ((uint32_t)(quad * 32) << 16), v);
        if (FOLD) {
          float v2[32];
          tmem_ld32(tmem + ab * acc_cols + LPB + ((uint32_t)(quad * 32) << 16), v2);
#pragma unroll
          for (int q = 0; q < 32; ++q) v[q] += v2[q];
        }
        const int64_t grow = (int64_t)t * BM + row;
        if (grow < mext[b]) {
          float* dst = y + (yoff[b] + grow) * LPB;
#pragma unroll
          for (int q = 0; q < 32; q += 4)
            *reinterpret_cast<float4*>(dst + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_acc_empty[ab]);
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

// ---------------------------------------------------------------------------
// test matrices
// ---------------------------------------------------------------------------
// blockIdx.y = g, the group of four columns 4g .. 4g + 3; a thread per row r (over all
// matrices' rows), its matrix found by binary search on roff.
__global__ void batched_draw_kernel(uint64_t seed, const int64_t* __restrict__ roff, int nb, int l,
                                    float* __restrict__ omega, __nv_bfloat16* __restrict__ xbf,
                                    int64_t ldx, const int64_t* __restrict__ xoff) {
  const int64_t nrows = roff[nb];
  const int g = blockIdx.y;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int b = find_matrix(roff, nb, r);
    const int64_t i = r - roff[b];
    float z[4] = {0.f, 0.f, 0.f, 0.f};
    if (4 * g < l) {
      const float4 v = gaussian4(seed_key(seed + (uint64_t)b), (uint32_t)g, (uint32_t)i, 0u);
      z[0] = v.x; z[1] = v.y; z[2] = v.z; z[3] = v.w;
    }
    // the float32 copy holds exactly the bfloat16 values the first pass multiplies with
    __nv_bfloat16 h[4];
    float f[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      h[q] = __float2bfloat16_rn(4 * g + q < l ? z[q] : 0.0f);
      f[q] = __bfloat162float(h[q]);
    }
    *reinterpret_cast<float4*>(omega + r * LPB + 4 * g) = make_float4(f[0], f[1], f[2], f[3]);
    if (xbf) {
      __nv_bfloat16* xb = xbf + xoff[b] + i;
#pragma unroll
      for (int q = 0; q < 4; ++q) xb[(int64_t)(4 * g + q) * ldx] = h[q];
    }
  }
}

// ---------------------------------------------------------------------------
// Cholesky QR, one CTA per matrix
// ---------------------------------------------------------------------------

// 32 x 32 Cholesky of S (+ shift, pivot floor) and inverse, by warp 0: lane r holds
// row r of L (a) and column r of X = L^-1 (x); entries above the diagonal of a are
// scratch.  Writes L into Ls (row-major, lower) and X into Xs.
__device__ __forceinline__ void chol32_warp(const float (*S)[LPB + 1], int l, float shift,
                                            float pfloor, float (*Ls)[LPB + 1],
                                            float (*Xs)[LPB + 1], uint32_t* status) {
  const int r = threadIdx.x & 31;
  float a[LPB], rpv[LPB];
#pragma unroll
  for (int j = 0; j < LPB; ++j) {
    float v = S[r][j];
    if (r >= l || j >= l) v = (r == j) ? 1.0f : 0.0f;   // identity beyond l
    else if (r == j) v += shift;
    a[j] = v;
  }
#pragma unroll
  for (int j = 0; j < LPB; ++j) {
    float d = __shfl_sync(0xffffffffu, a[j], j);
    if (j < l && !(d > pfloor)) {
      if (r == 0) set_status(status, isnan(d) ? ST_NONFINITE : ST_RANK_DEFICIENT);
      d = pfloor;
    }
    float rp = rsqrtf(d);
    rp = rp * fmaf(-0.5f * d * rp, rp, 1.5f);   // one Newton step for 1/sqrt(d)
    rpv[j] = rp;
    const float lij = (r == j) ? d * rp : (r > j ? a[j] * rp : 0.0f);
    a[j] = lij;
#pragma unroll
    for (int k = j + 1; k < LPB; ++k) a[k] = fmaf(-lij, __shfl_sync(0xffffffffu, lij, k), a[k]);
  }
  float x[LPB];
#pragma unroll
  for (int i = 0; i < LPB; ++i) {
    float v0 = 0.0f, v1 = 0.0f;
#pragma unroll
    for (int k = 0; k < i; ++k) {
      const float lik = __shfl_sync(0xffffffffu, a[k], i);
      if (k & 1) v1 = fmaf(lik, x[k], v1);
      else v0 = fmaf(lik, x[k], v0);
    }
    x[i] = (i > r) ? -(v0 + v1) * rpv[i] : (i == r ? rpv[i] : 0.0f);
  }
#pragma unroll
  for (int j = 0; j < LPB; ++j) Ls[r][j] = (j <= r) ? a[j] : 0.0f;
#pragma unroll
  for (int i = 0; i < LPB; ++i) Xs[i][r] = x[i];
}

// Cholesky-QR over 128-row units (matrix b, tile t; units of one matrix are consecutive,
// from ustart[b]): every step is one launch over all units of the batch, so the rows of
// all matrices are worked on in parallel instead of one CTA streaming each matrix.
//   bqr_gram_kernel  : the Gram of a unit's rows (staged in shared memory), a 32 x 32
//                      partial per unit;
//   bqr_chol_kernel  : one CTA per matrix: the sum of its units' partials in unit order
//                      (deterministic), the factor and its inverse by one warp in
//                      registers (shift on the first of three rounds, pivot floor), the
//                      running product of the R factors, and R^-1 for the apply;
//   bqr_apply_kernel : Q = Y R^-1 a thread per row, and the Gram partial of the new rows
//                      for the next round.
constexpr int kUnitRows = 128;
constexpr int kUnitThreads = 256;

// A unit's rows into shared memory (kUnitThreads threads): every thread's four 16-byte
// loads are issued before the first store, so they are in flight together.
__device__ __forceinline__ void bqr_stage(const float* __restrict__ src, int64_t row0, int nr,
                                          float (*ys)[LPB]) {
  constexpr int N = kUnitRows * (LPB / 4) / kUnitThreads;
  float4 v[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int e = threadIdx.x + k * kUnitThreads, rr = e >> 3;
    v[k] = rr < nr ? reinterpret_cast<const float4*>(src + (row0 + rr) * LPB)[e & 7] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int k = 0; k < N; ++k) reinterpret_cast<float4*>(&ys[0][0])[threadIdx.x + k * kUnitThreads] = v[k];
}

// Gram partial of the staged rows (NT threads, row r at ys + r YS): only the lower
// triangle of the l x l block is formed (the factorisation reads no more), as 4 x 4 tiles,
// L4 = ceil(l / 4) tile rows and L4 (L4 + 1) / 2 tiles; the threads form NG = NT / tiles
// row groups (12 at l = 24 and NT = 256), each thread one tile over its group's rows (two
// float4 reads per 16 FMAs).  The groups are summed in a fixed order through gp (NG x
// tiles x 16 floats, at most NT x 16), and the partial is written whole: zero above the
// diagonal tiles and beyond l.
template <int NT, int YS>
__device__ __forceinline__ void bqr_gram_tile(const float* ys, int nr, int l, float* gp,
                                              float* __restrict__ part) {
  const int l4 = (l + 3) >> 2;
  const int ntile = l4 * (l4 + 1) / 2;
  const int ng = NT / ntile;
  const int grp = threadIdx.x / ntile, t = threadIdx.x - grp * ntile;
  if (grp < ng) {
    int ti = 0, tt = t;
    while (tt > ti) { tt -= ti + 1; ++ti; }
    const int bi = 4 * ti, bj = 4 * tt;   // tt <= ti
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
#pragma unroll 4
    for (int rr = grp; rr < nr; rr += ng) {
      const float4 a = *reinterpret_cast<const float4*>(ys + rr * YS + bi);
      const float4 c = *reinterpret_cast<const float4*>(ys + rr * YS + bj);
      const float av[4] = {a.x, a.y, a.z, a.w}, cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], cv[j], acc[i][j]);
    }
    float* d = gp + (grp * ntile + t) * 16;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      *reinterpret_cast<float4*>(d + 4 * i) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < LPB * LPB; e += NT) {
    const int i = e >> 5, j = e & 31, ti = i >> 2, tj = j >> 2;
    float v = 0.0f;
    if (ti < l4 && tj <= ti) {
      const int off = (ti * (ti + 1) / 2 + tj) * 16 + (i & 3) * 4 + (j & 3);
      for (int g = 0; g < ng; ++g) v += gp[g * ntile * 16 + off];
    }
    part[e] = v;
  }
}

__global__ void __launch_bounds__(kUnitThreads) bqr_gram_kernel(const float* __restrict__ src,
                                                                const int64_t* __restrict__ roff,
                                                                const int2* __restrict__ units, int l,
                                                                float* __restrict__ part) {
  __shared__ __align__(16) float ys[kUnitRows][LPB];
  __shared__ __align__(16) float gp[kUnitThreads * 16];
  const int2 u = units[blockIdx.x];
  const int64_t row0 = roff[u.x] + (int64_t)u.y * kUnitRows;
  const int nr = (int)min((int64_t)kUnitRows, roff[u.x + 1] - row0);
  bqr_stage(src, row0, nr, ys);
  __syncthreads();
  bqr_gram_tile<kUnitThreads, LPB>(&ys[0][0], nr, l, gp, part + (size_t)blockIdx.x * LPB * LPB);
}

__global__ void __launch_bounds__(128) bqr_chol_kernel(const float* __restrict__ part,
                                                       const int* __restrict__ ustart, int l, float shift_on,
                                                       int racc_init, float* __restrict__ racc,
                                                       float* __restrict__ rinv, uint32_t* status) {
  __shared__ float S[LPB][LPB + 1];
  __shared__ float Ls[LPB][LPB + 1];
  __shared__ float Xs[LPB][LPB + 1];
  __shared__ float Ro[LPB][LPB + 1];
  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // every thread sums its 8 entries over the matrix's units in unit order, the loads of
  // four units (32) in flight together
  constexpr int kPer = LPB * LPB / 128;
  float v[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) v[q] = 0.0f;
  const int u0 = ustart[b], u1 = ustart[b + 1];
  int u = u0;
  for (; u + 4 <= u1; u += 4) {
    float w[4][kPer];
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
      for (int q = 0; q < kPer; ++q) w[d][q] = part[(size_t)(u + d) * LPB * LPB + tid + q * 128];
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
      for (int q = 0; q < kPer; ++q) v[q] += w[d][q];
  }
  for (; u < u1; ++u) {
    const float* pu = part + (size_t)u * LPB * LPB;
#pragma unroll
    for (int q = 0; q < kPer; ++q) v[q] += pu[tid + q * 128];
  }
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int e = tid + q * 128;
    S[e >> 5][e & 31] = v[q];
    Ro[e >> 5][e & 31] = racc[(size_t)b * LPB * LPB + e];
  }
  __syncthreads();
  if (warp == 0) {
    const float d = lane < l ? S[lane][lane] : 0.0f;
    float tr = warp_sum(d), mx = d;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (!isfinite(tr) && lane == 0) set_status(status, ST_NONFINITE);
    const float shift = shift_on * (float)l * kEpsF32 * tr;
    const float pfloor = fmaxf((float)l * kEpsF32 * mx, 1e-30f);
    chol32_warp(S, l, shift, pfloor, Ls, Xs, status);
  }
  __syncthreads();
  // R = L^T; the running product R Racc (or R itself on the first round), and R^-1 = X^T
  for (int e = tid; e < LPB * LPB; e += blockDim.x) {
    const int i = e >> 5, j = e & 31;
    float v = 0.0f;
    if (racc_init) {
      v = (j >= i) ? Ls[j][i] : 0.0f;
    } else {
      for (int c = i; c <= j; ++c) v = fmaf(Ls[c][i], Ro[c][j], v);
      if (j < i) v = 0.0f;
    }
    racc[(size_t)b * LPB * LPB + e] = (i < l && j < l) ? v : 0.0f;
    rinv[(size_t)b * LPB * LPB + e] = Xs[j][i];
  }
}

// Q = Y R^-1 over a unit, a thread per row (kApplyThreads = kUnitRows threads): the unit's
// rows are staged in shared memory by coalesced 16-byte loads (row stride 36 floats, so
// both these stores and a thread's reads of its own row are free of bank conflicts), a
// thread takes its row into registers and forms its row of Q with R^-1 read as float4
// broadcasts, summing only the triangle R^-1 has: column block c4 (4 columns) of Q sums
// rows 0 .. 4 c4 + 3 of R^-1, over the L4 = ceil(l / 4) blocks that can be nonzero (in row
// order, as the definition writes the sums).  The new rows replace the old in shared
// memory, leave by coalesced stores, and give the Gram partial of the next round.
constexpr int kApplyThreads = kUnitRows;
constexpr int kApplyCtasPerSm = 4;   // persistent apply: at most 53 KB of shared memory per CTA
static_assert(kUnitRows == kTileRows && LPB == kTileWidth, "units are the row tiles of batched_rows.cuh");

// With xbf, the new rows also go out as the next pass's operand, transposed bfloat16 (the
// layout of batched_to_bf16t_kernel, written from the registers that hold them).
// Persistent: a CTA takes units blockIdx.x, + gridDim.x, ...; while it works one unit, the
// rows and the R^-1 of its next unit are already being copied into the other half of a
// double buffer (cp.async), so the unit's loads are not waited for between units.
// Dynamic shared memory: apply_smem<L4>() bytes.
template <int L4>
constexpr size_t apply_smem() {
  return (size_t)(2 * kUnitRows * kRowStride + 2 * (4 * L4) * (4 * L4) + kApplyThreads * 16) * sizeof(float);
}

template <int L4>
__global__ void __launch_bounds__(kApplyThreads) bqr_apply_kernel(const float* __restrict__ src,
                                                                  float* __restrict__ dst,
                                                                  const int64_t* __restrict__ roff,
                                                                  const int2* __restrict__ units, int nunits, int l,
                                                                  const float* __restrict__ rinv,
                                                                  float* __restrict__ part,
                                                                  __nv_bfloat16* __restrict__ xbf, int64_t ldx,
                                                                  const int64_t* __restrict__ xoff, int split) {
  constexpr int LC = 4 * L4;
  extern __shared__ __align__(16) float dsm[];
  // staged rows of two units, then R^-1 (LC x LC) of two units, then the Gram scratch
  auto ysb = [&](int b) { return dsm + b * (kUnitRows * kRowStride); };
  auto rsb = [&](int b) { return dsm + 2 * kUnitRows * kRowStride + b * (LC * LC); };
  float* gp = dsm + 2 * kUnitRows * kRowStride + 2 * LC * LC;
  const int t = threadIdx.x;
  auto issue = [&](int ui, int b) {
    const int2 u = units[ui];
    const int64_t row0 = roff[u.x] + (int64_t)u.y * kUnitRows;
    const int nr = (int)min((int64_t)kUnitRows, roff[u.x + 1] - row0);
    stage_tile_async<L4>(src, row0, nr, ysb(b));
    for (int e = t; e < LC * L4; e += kApplyThreads) {
      const int i = e / L4, c4 = e - i * L4;
      cp_async16(rsb(b) + i * LC + 4 * c4, rinv + (size_t)u.x * LPB * LPB + i * LPB + 4 * c4, true);
    }
  };
  int ui = blockIdx.x;
  if (ui >= nunits) return;
  issue(ui, 0);
  cp_async_commit();
  for (int b = 0; ui < nunits; ui += gridDim.x, b ^= 1) {
    if (ui + (int)gridDim.x < nunits) issue(ui + gridDim.x, b ^ 1);
    cp_async_commit();
    cp_async_wait<1>();   // this unit's copies have landed; the next unit's may still fly
    __syncthreads();
    float* ys = ysb(b);
    const float* rs = rsb(b);
    const int2 u = units[ui];
    const int64_t row0 = roff[u.x] + (int64_t)u.y * kUnitRows;
    const int nr = (int)min((int64_t)kUnitRows, roff[u.x + 1] - row0);
    float y[LC];
    load_row<L4>(ys, t, y);
#pragma unroll
    for (int c4 = 0; c4 < L4; ++c4) {
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int i = 0; i < 4 * c4 + 4; ++i) {
        const float4 r = *reinterpret_cast<const float4*>(rs + i * LC + 4 * c4);
        acc.x = fmaf(y[i], r.x, acc.x);
        acc.y = fmaf(y[i], r.y, acc.y);
        acc.z = fmaf(y[i], r.z, acc.z);
        acc.w = fmaf(y[i], r.w, acc.w);
      }
      // row t of the staged tile is read by this thread alone (its y is in registers)
      *reinterpret_cast<float4*>(ys + t * kRowStride + 4 * c4) = acc;
      if (xbf && t < nr) {
        __nv_bfloat16* xb = xbf + xoff[u.x] + (int64_t)u.y * kUnitRows + t;
        const float a4[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const __nv_bfloat16 hi = __float2bfloat16_rn(a4[i]);
          xb[(int64_t)(4 * c4 + i) * ldx] = hi;
          if (split) xb[(int64_t)(LPB + 4 * c4 + i) * ldx] = __float2bfloat16_rn(a4[i] - __bfloat162float(hi));
        }
      }
    }
    if (xbf && t < nr) {   // the zero columns beyond 4 L4
      __nv_bfloat16* xb = xbf + xoff[u.x] + (int64_t)u.y * kUnitRows + t;
      const __nv_bfloat16 z = __float2bfloat16_rn(0.0f);
      for (int c = LC; c < LPB; ++c) {
        xb[(int64_t)c * ldx] = z;
        if (split) xb[(int64_t)(LPB + c) * ldx] = z;
      }
    }
    __syncthreads();
    store_tile<L4>(ys, nr, dst, row0, LPB);   // the new rows out, zeros beyond column 4 L4
    if (part) bqr_gram_tile<kApplyThreads, kRowStride>(ys, nr, l, gp, part + (size_t)ui * LPB * LPB);
    __syncthreads();   // this unit's buffers are free for the copies issued next iteration
  }
}

// basis rows (concatenated, LPB wide) -> transposed bfloat16 operand (LPB x sum K); one CTA
// per matrix, a thread per row (row reads from L1, column writes coalesced across threads)
__global__ void __launch_bounds__(256) batched_to_bf16t_kernel(const float* __restrict__ q,
                                                               const int64_t* __restrict__ roff,
                                                               __nv_bfloat16* __restrict__ xbf,
                                                               int64_t ldx,
                                                               const int64_t* __restrict__ xoff,
                                                               int split) {
  const int b = blockIdx.x;
  const int64_t r0 = roff[b], rows = roff[b + 1] - r0;
  __nv_bfloat16* xb = xbf + xoff[b];
  for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) {
    const float4* src = reinterpret_cast<const float4*>(q + (r0 + i) * LPB);
#pragma unroll
    for (int c4 = 0; c4 < LPB / 4; ++c4) {
      const float4 v4 = src[c4];
      const float v[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int c = 4 * c4 + t;
        const __nv_bfloat16 hi = __float2bfloat16_rn(v[t]);
        xb[(int64_t)c * ldx + i] = hi;
        if (split) xb[(int64_t)(LPB + c) * ldx + i] = __float2bfloat16_rn(v[t] - __bfloat162float(hi));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// one-sided Jacobi of the l x l matrices (x_b or x_b^T), one CTA per matrix
// ---------------------------------------------------------------------------
constexpr int kJThreads = 256;   // 8 warps: a half-warp per column pair of a round (16 pairs)

__global__ void __launch_bounds__(kJThreads) batched_jacobi_kernel(
    const float* __restrict__ x, int transposed, int l, float* __restrict__ ut,
    float* __restrict__ sig, float* __restrict__ w, uint32_t* status, uint32_t* info, float tol) {
  __shared__ float Xc[LPB][LPB + 1];   // column c of X in Xc[c][*]
  __shared__ float Jc[LPB][LPB + 1];
  __shared__ float s_sig[LPB];
  __shared__ int s_rot;
  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* xb = x + (size_t)b * LPB * LPB;
  for (int e = tid; e < LPB * LPB; e += kJThreads) {
    const int c = e / LPB, r = e % LPB;
    float v = 0.0f;
    if (r < l && c < l) v = transposed ? xb[c * LPB + r] : xb[r * LPB + c];
    Xc[c][r] = v;
    Jc[c][r] = (c < l && r == c) ? 1.0f : 0.0f;
  }
  if (tid == 0) s_rot = 0;
  __syncthreads();
  const int le = l + (l & 1);
  // a half-warp per pair (two per warp): lane h of it holds rows h and h + 16 of both
  // columns, so the three sums take four shuffle levels
  const int half = lane >> 4, hl = lane & 15;
  const int pr = 2 * warp + half;   // the pair of the round this half-warp takes
  int sweep = 0;
  for (; sweep < 40; ++sweep) {
    for (int round = 0; round < le - 1; ++round) {
      if (pr < le / 2) {
        const int p = pr == 0 ? 0 : ((pr - 1 + round) % (le - 1)) + 1;
        const int kq = le - 1 - pr;
        const int q = kq == 0 ? 0 : ((kq - 1 + round) % (le - 1)) + 1;
        if (p < l && q < l) {
          const float u0 = Xc[p][hl], u1 = Xc[p][hl + 16], v0 = Xc[q][hl], v1 = Xc[q][hl + 16];
          float a = fmaf(u0, u0, u1 * u1), bb = fmaf(v0, v0, v1 * v1), g = fmaf(u0, v0, u1 * v1);
#pragma unroll
          for (int o = 8; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            bb += __shfl_xor_sync(0xffffffffu, bb, o);
            g += __shfl_xor_sync(0xffffffffu, g, o);
          }
          if (g != 0.0f && fabsf(g) > tol * sqrtf(a * bb)) {
            const float zeta = __fdividef(bb - a, 2.0f * g);
            const float az = fabsf(zeta);
            float t = (az > 1e18f) ? __fdividef(0.5f, az) : __fdividef(1.0f, az + sqrtf(fmaf(az, az, 1.0f)));
            t = copysignf(t, zeta);
            if (zeta == 0.0f) t = 1.0f;
            const float w2 = fmaf(t, t, 1.0f);
            float c = rsqrtf(w2);
            c = c * fmaf(-0.5f * w2, c * c, 1.5f);
            const float sn = c * t, tau = __fdividef(sn, 1.0f + c);
            Xc[p][hl] = u0 - sn * fmaf(tau, u0, v0);
            Xc[q][hl] = v0 + sn * fmaf(-tau, v0, u0);
            Xc[p][hl + 16] = u1 - sn * fmaf(tau, u1, v1);
            Xc[q][hl + 16] = v1 + sn * fmaf(-tau, v1, u1);
            const float j0 = Jc[p][hl], j1 = Jc[p][hl + 16], k0 = Jc[q][hl], k1 = Jc[q][hl + 16];
            Jc[p][hl] = j0 - sn * fmaf(tau, j0, k0);
            Jc[q][hl] = k0 + sn * fmaf(-tau, k0, j0);
            Jc[p][hl + 16] = j1 - sn * fmaf(tau, j1, k1);
            Jc[q][hl + 16] = k1 + sn * fmaf(-tau, k1, j1);
            if (hl == 0) s_rot = 1;
          }
        }
      }
      __syncthreads();
    }
    const int rot = s_rot;
    __syncthreads();
    if (tid == 0) s_rot = 0;
    __syncthreads();
    if (!rot) break;
  }
  if (tid == 0) {
    if (sweep == 40) set_status(status, ST_JACOBI_NOCONV);
    if (info) atomicMax(info, (uint32_t)(sweep + 1));
  }
  if (warp < LPB) {
    for (int c = warp; c < LPB; c += kJThreads / 32) {
      const float v = Xc[c][lane];
      const float s2 = warp_sum(v * v);
      if (lane == 0) s_sig[c] = c < l ? sqrtf(s2) : -1.0f;
    }
  }
  __syncthreads();
  float* ub = ut + (size_t)b * LPB * LPB;
  float* wb = w + (size_t)b * LPB * LPB;
  for (int e = tid; e < LPB * LPB; e += kJThreads) {
    const int r = e / LPB, c = e % LPB;
    if (r >= l || c >= l) { ub[e] = 0.0f; wb[e] = 0.0f; }
  }
  for (int c = warp; c < l; c += kJThreads / 32) {
    const float sc = s_sig[c];
    int rk = 0;
    for (int c2 = 0; c2 < l; ++c2) {
      const float s2 = s_sig[c2];
      rk += (s2 > sc || (s2 == sc && c2 < c)) ? 1 : 0;
    }
    const float inv = sc > 0.0f ? 1.0f / sc : 0.0f;
    if (lane < l) {
      ub[lane * LPB + rk] = Xc[c][lane] * inv;
      wb[lane * LPB + rk] = Jc[c][lane];
    }
    if (lane == 0) sig[(size_t)b * LPB + rk] = sc;
  }
}

// out rows (concatenated, ldo wide) = Q_b rows times the first `cols` columns of the
// per-matrix LPB x LPB block small_b (ld LPB): out[r][c] = sum_j Q[r][j] small_b[j][c]
// for c < valid, 0 for valid <= c < cols; one CTA per matrix, a warp per row
// One CTA per (matrix, block of kLiftRows rows), a thread per row: the rows of Q_b (their
// first l columns, the others are zero) staged in shared memory by coalesced loads, a
// thread's row into registers, the small matrix's first 4 ceil(l / 4) rows in shared memory
// read as float4 broadcasts (columns >= valid read as zero), the sums in row order; the
// output rows go back through shared memory and leave by coalesced stores when vec (cols
// and ldo multiples of 4, out 16-byte aligned), else a thread writes its own row.
constexpr int kLiftRows = 128;

template <int L4>
__global__ void __launch_bounds__(kLiftRows) batched_lift_kernel(const float* __restrict__ q,
                                                                 const int64_t* __restrict__ roff,
                                                                 const float* __restrict__ small, int cols,
                                                                 int valid, float* __restrict__ out, int ldo,
                                                                 int vec) {
  static_assert(kLiftRows == kUnitRows, "the lift stages rows like a Cholesky-QR unit");
  constexpr int LC = 4 * L4;
  __shared__ __align__(16) float ys[kLiftRows * kRowStride];
  __shared__ __align__(16) float Ss[LC][LPB];
  const int b = blockIdx.x;
  const int64_t r_begin = roff[b] + (int64_t)blockIdx.y * kLiftRows;
  const int64_t r_end = min(roff[b + 1], r_begin + kLiftRows);
  if (r_begin >= r_end) return;
  const int nr = (int)(r_end - r_begin);
  const int t = threadIdx.x;
  stage_tile<L4>(q, r_begin, nr, ys);
  for (int e = t; e < LC * LPB; e += kLiftRows) {
    const int c = e % LPB;
    Ss[e / LPB][c] = c < valid ? small[(size_t)b * LPB * LPB + e] : 0.0f;
  }
  __syncthreads();
  float y[LC];
  load_row<L4>(ys, t, y);
  const int n4 = (cols + 3) / 4;
  for (int c4 = 0; c4 < n4; ++c4) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < LC; ++j) {
      const float4 sv = *reinterpret_cast<const float4*>(&Ss[j][4 * c4]);
      acc.x = fmaf(y[j], sv.x, acc.x);
      acc.y = fmaf(y[j], sv.y, acc.y);
      acc.z = fmaf(y[j], sv.z, acc.z);
      acc.w = fmaf(y[j], sv.w, acc.w);
    }
    if (vec) {
      *reinterpret_cast<float4*>(ys + t * kRowStride + 4 * c4) = acc;   // this thread's row only
    } else if (t < nr) {
      const float a4[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (4 * c4 + i < cols) out[(r_begin + t) * ldo + 4 * c4 + i] = a4[i];
    }
  }
  if (!vec) return;
  __syncthreads();
  for (int e = t; e < nr * n4; e += kLiftRows) {
    const int rr = e / n4, c4 = e - rr * n4;
    *reinterpret_cast<float4*>(out + (r_begin + rr) * ldo + 4 * c4) =
        *reinterpret_cast<const float4*>(ys + rr * kRowStride + 4 * c4);
  }
}

unsigned grid_for(int64_t n) {
  const int64_t b = cdiv(n, 256);
  return (unsigned)(b < 16 * kNumSMs ? (b < 1 ? 1 : b) : 16 * kNumSMs);
}

}  // namespace

size_t batched_tc_smem(int stages, int fold) {
  return (size_t)stages * (BM * BK * 2 + (fold ? 2 : 1) * LPB * BK * 2) + 1024;
}

template <int L4>
cudaError_t prep_apply() {
  return cudaFuncSetAttribute(bqr_apply_kernel<L4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)apply_smem<L4>());
}

cudaError_t prepare_batched() {
  {
    cudaError_t e;
    if ((e = prep_apply<1>()) != cudaSuccess || (e = prep_apply<2>()) != cudaSuccess ||
        (e = prep_apply<3>()) != cudaSuccess || (e = prep_apply<4>()) != cudaSuccess ||
        (e = prep_apply<5>()) != cudaSuccess || (e = prep_apply<6>()) != cudaSuccess ||
        (e = prep_apply<7>()) != cudaSuccess || (e = prep_apply<8>()) != cudaSuccess)
      return e;
  }
  cudaError_t e;
  const int s0 = (int)batched_tc_smem(kBatchedStages, 0), s1 = (int)batched_tc_smem(kBatchedStages, 1);
  if ((e = cudaFuncSetAttribute(batched_tc_kernel<0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, s0)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(batched_tc_kernel<1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, s0)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(batched_tc_kernel<0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, s1)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(batched_tc_kernel<1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, s1);
}

cudaError_t launch_batched_tc(int mode, int fold, const void* maps, const void* map_x,
                              const int2* units, int nunits, const int64_t* kext, const int64_t* mext,
                              const int64_t* xoff, const int64_t* yoff, float* y, int grid,
                              uint32_t* status, cudaStream_t st, int stages) {
  if (nunits <= 0) return cudaSuccess;
  if (stages < 2 || stages > kBatchedStages) return cudaErrorInvalidValue;
  const CUtensorMap* mp = static_cast<const CUtensorMap*>(maps);
  const CUtensorMap& mx = *static_cast<const CUtensorMap*>(map_x);
  const size_t sm = batched_tc_smem(stages, fold);
  if (grid > nunits) grid = nunits;
#define RSVD_BTC(MO, FO)                                                                        \
  batched_tc_kernel<MO, FO><<<grid, kBThreads, sm, st>>>(mp, mx, units, nunits, kext, mext, xoff, \
                                                         yoff, y, stages, status)
  if (mode == 0 && !fold) RSVD_BTC(0, 0);
  else if (mode == 0) RSVD_BTC(0, 1);
  else if (!fold) RSVD_BTC(1, 0);
  else RSVD_BTC(1, 1);
#undef RSVD_BTC
  return cudaGetLastError();
}

cudaError_t launch_batched_draw(uint64_t seed, const int64_t* roff, int nb, int64_t total_rows, int l,
                                float* omega, __nv_bfloat16* xbf, int64_t ldx, const int64_t* xoff,
                                cudaStream_t st) {
  const dim3 grid(grid_for(total_rows), LPB / 4);
  batched_draw_kernel<<<grid, 256, 0, st>>>(seed, roff, nb, l, omega, xbf, ldx, xoff);
  return cudaGetLastError();
}

cudaError_t launch_batched_cholqr(const float* yin, float* qout, const int64_t* roff, int nb, int l,
                                  int rounds, int shift_first, float* rout, float* rinv, const int2* units,
                                  int nunits, const int* ustart, float* part, uint32_t* status, cudaStream_t st,
                                  __nv_bfloat16* xbf, int64_t ldx, const int64_t* xoff, int split) {
  if (nunits <= 0 || rounds < 1) return cudaErrorInvalidValue;
  bqr_gram_kernel<<<nunits, kUnitThreads, 0, st>>>(yin, roff, units, l, part);
  for (int r = 0; r < rounds; ++r) {
    bqr_chol_kernel<<<nb, 128, 0, st>>>(part, ustart, l, (shift_first && r == 0) ? 1.0f : 0.0f, r == 0 ? 1 : 0,
                                        rout, rinv, status);
    const float* yr = r == 0 ? yin : qout;
    const bool last = r + 1 == rounds;
    float* pr = last ? nullptr : part;
    __nv_bfloat16* xo = last ? xbf : nullptr;
    const int grid = nunits < kApplyCtasPerSm * kNumSMs ? nunits : kApplyCtasPerSm * kNumSMs;
    switch ((l + 3) / 4) {
#define RSVD_BQR_APPLY(L4)                                                                          \
  case L4:                                                                                         \
    bqr_apply_kernel<L4><<<grid, kApplyThreads, apply_smem<L4>(), st>>>(yr, qout, roff, units, nunits, \
                                                                       l, rinv, pr, xo, ldx, xoff,   \
                                                                       split);                       \
    break;
      RSVD_BQR_APPLY(1) RSVD_BQR_APPLY(2) RSVD_BQR_APPLY(3) RSVD_BQR_APPLY(4)
      RSVD_BQR_APPLY(5) RSVD_BQR_APPLY(6) RSVD_BQR_APPLY(7) RSVD_BQR_APPLY(8)
#undef RSVD_BQR_APPLY
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_batched_to_bf16t(const float* q, const int64_t* roff, int nb, int64_t total_rows,
                                    __nv_bfloat16* xbf, int64_t ldx, const int64_t* xoff, int split,
                                    cudaStream_t st) {
  (void)total_rows;
  batched_to_bf16t_kernel<<<nb, 256, 0, st>>>(q, roff, xbf, ldx, xoff, split);
  return cudaGetLastError();
}

cudaError_t launch_batched_jacobi(const float* x, int transposed, int l, int nb, float* ut, float* sig,
                                  float* w, uint32_t* status, uint32_t* info, cudaStream_t st) {
  const float tol = 8.0f * sqrtf((float)l) * kEpsF32;
  batched_jacobi_kernel<<<nb, kJThreads, 0, st>>>(x, transposed, l, ut, sig, w, status, info, tol);
  return cudaGetLastError();
}

cudaError_t launch_batched_lift(const float* q, const int64_t* roff, int nb, int64_t max_rows, int l,
                                const float* small, int cols, int valid, float* out, int ldo,
                                cudaStream_t st) {
  if (cols > LPB || l < 1 || l > LPB || max_rows < 1 || cdiv(max_rows, kLiftRows) > 65535)
    return cudaErrorInvalidValue;
  const int vec = (cols % 4 == 0 && ldo % 4 == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0) ? 1 : 0;
  // blocks of kLiftRows rows per matrix, as many as the tallest matrix needs
  const dim3 grid((unsigned)nb, (unsigned)cdiv(max_rows, kLiftRows));
  switch ((l + 3) / 4) {
#define RSVD_LIFT_CASE(L4)                                                                               \
  case L4:                                                                                              \
    batched_lift_kernel<L4><<<grid, kLiftRows, 0, st>>>(q, roff, small, cols, valid, out, ldo, vec); \
    break;
    RSVD_LIFT_CASE(1) RSVD_LIFT_CASE(2) RSVD_LIFT_CASE(3) RSVD_LIFT_CASE(4)
    RSVD_LIFT_CASE(5) RSVD_LIFT_CASE(6) RSVD_LIFT_CASE(7) RSVD_LIFT_CASE(8)
#undef RSVD_LIFT_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace rsvd
