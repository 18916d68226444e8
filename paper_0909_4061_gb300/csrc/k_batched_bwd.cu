// Backward pass of the batched randomized SVD: the gradient of
//     L = sum_b ||A_b - U_b S_b V_b^T||_F^2 + sum_b sum_{i<=k} sigma_{b,i}
// through the map A -> (U, S, V) of Algorithm 4.4 + Algorithm 5.1 with the test
// matrices held fixed (reverse mode, per matrix).
//
// Forward, per matrix: Y_0 = A Omega = Q_0 R_0; for j = 1..q: A^T Q_{j-1} = Qt_j Rt_j,
// A Qt_j = Q_j R_j; B = Q^T A = Ut Sig Vb^T (Q = Q_q, Vb = Q_B W); U = Q Ut_k, V = Vb_k.
// Reverse:
//   * with the SVD of B exact, U^T (A - U S V^T) = 0, so dL/dV = 0, dL/dsigma_i = 1 and
//     Q^T dL/dU = 0: the SVD adjoint leaves dL/dB = Ut_k V^T, and
//       dL/dQ = dL/dU Ut_k^T + A (dL/dB)^T = (A V (I - 2 S) + 2 U S^2) Ut_k^T,
//     while the direct terms give 2 (A - U S V^T) + Q dL/dB = 2 A + U (I - 2 S) V^T;
//   * each QR step Y = Q R (Cholesky QR computes the unique Q, R with diag R > 0) maps
//     dL/dQ to dL/dY = (dL/dQ + Q copyltu(M)) R^-T with M = -(dL/dQ)^T Q, copyltu taking
//     the lower triangle and its mirror (no dependence on R downstream);
//   * a product Y = A X contributes dL/dY X^T to dL/dA and A^T dL/dY to dL/dX (the next
//     pass over A going down the chain); A^T X likewise.
// So dL/dA = 2 A + L R^T with L = [U (I - 2S) | dY_q | Q_{q-1} | ... | dY_0] and
// R = [V | Qt_q | dZ_q | ... | Omega]: q + 1 ... passes over A for A V and the chain,
// then one kernel that reads A and writes dL/dA.
#include <cuda.h>

#include "common.cuh"
#include "kernels_batched.cuh"
#include "tc_ptx.cuh"

namespace rsvd {
namespace {

using namespace tcx;

constexpr int LPB = 32;

// Row kernels of the backward over the 128-row units of the Cholesky-QR (one matrix per
// unit): the unit's rows and the matrix's 32 x 32 factors are staged in shared memory
// (coalesced), a warp takes a row at a time with lane = column, holding the column / row
// of each factor it needs in registers and reading the row as float4 broadcasts; results
// leave through the staging buffer, coalesced.
constexpr int kUR = 128;   // rows per unit
constexpr int kUT = 256;   // threads per unit block

__device__ __forceinline__ void unit_rows(const int64_t* __restrict__ roff, int2 u, int64_t* row0, int* nr) {
  *row0 = roff[u.x] + (int64_t)u.y * kUR;
  *nr = (int)min((int64_t)kUR, roff[u.x + 1] - *row0);
}

// (kUT threads; every thread's loads are issued before its first store, so they are in
// flight together)
__device__ __forceinline__ void unit_stage(const float* __restrict__ src, int64_t row0, int nr,
                                           float (*ys)[LPB]) {
  constexpr int N = kUR * (LPB / 4) / kUT;
  float4 v[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int e = threadIdx.x + k * kUT, rr = e >> 3;
    v[k] = rr < nr ? reinterpret_cast<const float4*>(src + (row0 + rr) * LPB)[e & 7] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int k = 0; k < N; ++k) reinterpret_cast<float4*>(&ys[0][0])[threadIdx.x + k * kUT] = v[k];
}

// a 32 x 32 factor into shared memory (rows padded to 33 floats: column and row reads
// by lane are both conflict-free)
__device__ __forceinline__ void unit_small(const float* __restrict__ src, float (*ms)[LPB + 1]) {
  constexpr int N = LPB * LPB / kUT;
  float v[N];
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = src[threadIdx.x + k * kUT];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int e = threadIdx.x + k * kUT;
    ms[e >> 5][e & 31] = v[k];
  }
}

// sum_j y_j w[j] for the row y in shared memory (float4 broadcasts), w in registers
__device__ __forceinline__ float row_dot(const float* __restrict__ y, const float (&w)[LPB]) {
  const float4* y4 = reinterpret_cast<const float4*>(y);
  float v0 = 0.0f, v1 = 0.0f;
#pragma unroll
  for (int i4 = 0; i4 < LPB / 4; ++i4) {
    const float4 a = y4[i4];
    v0 = fmaf(a.x, w[4 * i4], v0);
    v1 = fmaf(a.y, w[4 * i4 + 1], v1);
    v0 = fmaf(a.z, w[4 * i4 + 2], v0);
    v1 = fmaf(a.w, w[4 * i4 + 3], v1);
  }
  return v0 + v1;
}

// t_c = P[r][c] (1 - 2 s_c) + 2 s_c^2 u_c with u = Q[r] Ut; gQ[r][i] = sum_{c<k} t_c Ut[i][c];
// ublk[r][c] = u_c (1 - 2 s_c) for c < k, zero beyond (the first left factor U (I - 2S)).
__global__ void __launch_bounds__(kUT) bwd_gq_kernel(const float* __restrict__ P, const float* __restrict__ Q,
                                                     const int64_t* __restrict__ roff,
                                                     const int2* __restrict__ units,
                                                     const float* __restrict__ ut, const float* __restrict__ sig,
                                                     int k, float* __restrict__ gq, float* __restrict__ ublk,
                                                     int ldu) {
  __shared__ __align__(16) float qs[kUR][LPB];
  __shared__ __align__(16) float ps[kUR][LPB];
  __shared__ __align__(16) float tb[kUT / 32][LPB];
  __shared__ float Us[LPB][LPB + 1];
  const int2 u = units[blockIdx.x];
  int64_t row0;
  int nr;
  unit_rows(roff, u, &row0, &nr);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unit_stage(Q, row0, nr, qs);
  unit_stage(P, row0, nr, ps);
  unit_small(ut + (size_t)u.x * LPB * LPB, Us);
  const float s = lane < k ? sig[(size_t)u.x * LPB + lane] : 0.0f;
  const float c1 = 1.0f - 2.0f * s, c2 = 2.0f * s * s;
  __syncthreads();
  float ucol[LPB], urow[LPB];
#pragma unroll
  for (int j = 0; j < LPB; ++j) {
    ucol[j] = Us[j][lane];   // Ut[j][lane]
    urow[j] = Us[lane][j];   // Ut[lane][j]
  }
  for (int rr = warp; rr < nr; rr += kUT / 32) {
    const float uc = row_dot(qs[rr], ucol);
    const float t = lane < k ? fmaf(ps[rr][lane], c1, c2 * uc) : 0.0f;
    tb[warp][lane] = t;
    __syncwarp();
    const float g = row_dot(tb[warp], urow);
    __syncwarp();   // the warp's rows and its tb row are read before they are overwritten
    qs[rr][lane] = g;
    ps[rr][lane] = lane < k ? uc * c1 : 0.0f;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nr * LPB; e += blockDim.x) {
    const int rr = e >> 5, c = e & 31;
    gq[(row0 + rr) * LPB + c] = qs[rr][c];
    ublk[(row0 + rr) * ldu + c] = ps[rr][c];
  }
}

// gY = (gQ + Q N) R^-T per row: lane j forms w_j = gQ[r][j] + sum_t Q[r][t] N[t][j] (column
// j of N in registers); lane i then gY[r][i] = sum_j w_j Rinv[i][j] (row i of R^-1).
__global__ void __launch_bounds__(kUT) bwd_qr_apply_kernel(const float* __restrict__ Q,
                                                           const float* __restrict__ gQ,
                                                           const int64_t* __restrict__ roff,
                                                           const int2* __restrict__ units,
                                                           const float* __restrict__ N,
                                                           const float* __restrict__ Rinv,
                                                           float* __restrict__ gY) {
  __shared__ __align__(16) float qs[kUR][LPB];
  __shared__ __align__(16) float gs[kUR][LPB];
  __shared__ __align__(16) float wb[kUT / 32][LPB];
  __shared__ float Ns[LPB][LPB + 1];
  __shared__ float Rs[LPB][LPB + 1];
  const int2 u = units[blockIdx.x];
  int64_t row0;
  int nr;
  unit_rows(roff, u, &row0, &nr);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unit_stage(Q, row0, nr, qs);
  unit_stage(gQ, row0, nr, gs);
  unit_small(N + (size_t)u.x * LPB * LPB, Ns);
  unit_small(Rinv + (size_t)u.x * LPB * LPB, Rs);
  __syncthreads();
  float ncol[LPB], rrow[LPB];
#pragma unroll
  for (int j = 0; j < LPB; ++j) {
    ncol[j] = Ns[j][lane];   // N[j][lane]
    rrow[j] = Rs[lane][j];   // Rinv[lane][j]
  }
  for (int rr = warp; rr < nr; rr += kUT / 32) {
    const float w = gs[rr][lane] + row_dot(qs[rr], ncol);
    wb[warp][lane] = w;
    __syncwarp();
    const float g = row_dot(wb[warp], rrow);
    __syncwarp();
    qs[rr][lane] = g;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nr * (LPB / 4); e += blockDim.x)
    reinterpret_cast<float4*>(gY + row0 * LPB)[e] = reinterpret_cast<const float4*>(&qs[0][0])[e];
}

// C_u = sum over the rows of a Cholesky-QR unit (matrix b, 128-row tile) of gQ[r][i] Q[r][j]:
// the partial of gQ^T Q, 256 threads in four row groups with 4 x 4 register blocks (two
// float4 reads per 16 FMAs), the groups summed in a fixed order.
constexpr int kCrossRows = 128;

__global__ void __launch_bounds__(256) bwd_cross_kernel(const float* __restrict__ gQ, const float* __restrict__ Q,
                                                        const int64_t* __restrict__ roff,
                                                        const int2* __restrict__ units, float* __restrict__ part) {
  __shared__ __align__(16) float gs[kCrossRows][LPB];
  __shared__ __align__(16) float qs[kCrossRows][LPB];
  __shared__ float gp[4][LPB * LPB / 4];   // one quarter of G per row group at a time
  const int2 u = units[blockIdx.x];
  const int64_t row0 = roff[u.x] + (int64_t)u.y * kCrossRows;
  const int nr = (int)min((int64_t)kCrossRows, roff[u.x + 1] - row0);
  for (int e = threadIdx.x; e < kCrossRows * (LPB / 4); e += blockDim.x) {
    const int rr = e >> 3;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    reinterpret_cast<float4*>(&gs[0][0])[e] = rr < nr ? reinterpret_cast<const float4*>(gQ + (row0 + rr) * LPB)[e & 7] : z;
    reinterpret_cast<float4*>(&qs[0][0])[e] = rr < nr ? reinterpret_cast<const float4*>(Q + (row0 + rr) * LPB)[e & 7] : z;
  }
  __syncthreads();
  const int grp = threadIdx.x >> 6, gt = threadIdx.x & 63;
  const int bi = (gt >> 3) * 4, bj = (gt & 7) * 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
  for (int rr = grp; rr < nr; rr += 4) {
    const float4 x = *reinterpret_cast<const float4*>(&gs[rr][bi]);
    const float4 y = *reinterpret_cast<const float4*>(&qs[rr][bj]);
    const float xv[4] = {x.x, x.y, x.z, x.w}, yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xv[i], yv[j], acc[i][j]);
  }
  // the four groups' blocks summed through shared memory, one row quarter of C at a time
  float* pu = part + (size_t)blockIdx.x * LPB * LPB;
  for (int qtr = 0; qtr < 4; ++qtr) {
    __syncthreads();
    if ((bi >> 3) == qtr) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) gp[grp][(bi - 8 * qtr + i) * LPB + bj + j] = acc[i][j];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < LPB * LPB / 4; e += blockDim.x)
      pu[qtr * (LPB * LPB / 4) + e] = (gp[0][e] + gp[1][e]) + (gp[2][e] + gp[3][e]);
  }
}

// per matrix: C = the sum of its units' partials (in unit order), N = copyltu(-C); Rinv =
// R^-1 from R^T = L lower: warp 0, lane r holds row r of L, X = L^-1 by columns.
__global__ void __launch_bounds__(128) bwd_qr_small_kernel(const float* __restrict__ part,
                                                           const int* __restrict__ ustart, int l,
                                                           const float* __restrict__ R, float* __restrict__ N,
                                                           float* __restrict__ Rinv) {
  __shared__ float C[LPB][LPB + 1];
  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kPer = LPB * LPB / 128;
  float v[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) v[q] = 0.0f;
  for (int u = ustart[b]; u < ustart[b + 1]; ++u) {
    const float* pu = part + (size_t)u * LPB * LPB;
#pragma unroll
    for (int q = 0; q < kPer; ++q) v[q] += pu[tid + q * 128];
  }
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int e = tid + q * 128;
    C[e >> 5][e & 31] = v[q];   // C(i, j) = sum_r gQ[r][i] Q[r][j]
  }
  __syncthreads();
  float* Nb = N + (size_t)b * LPB * LPB;
  for (int e = tid; e < LPB * LPB; e += blockDim.x) {
    const int i = e / LPB, j = e % LPB;
    Nb[e] = -(i >= j ? C[i][j] : C[j][i]);
  }
  if (warp == 0) {
    const float* Rb = R + (size_t)b * LPB * LPB;
    const int r = lane;
    float a[LPB];
#pragma unroll
    for (int j = 0; j < LPB; ++j) {
      float v = (j <= r) ? Rb[j * LPB + r] : 0.0f;   // L(r, j) = R(j, r)
      if (r >= l || j >= l) v = (r == j) ? 1.0f : 0.0f;
      a[j] = v;
    }
    float x[LPB];
#pragma unroll
    for (int i = 0; i < LPB; ++i) {
      const float lii = __shfl_sync(0xffffffffu, a[i], i);
      const float rinv = 1.0f / lii;
      float v0 = 0.0f, v1 = 0.0f;
#pragma unroll
      for (int kk = 0; kk < i; ++kk) {
        const float lik = __shfl_sync(0xffffffffu, a[kk], i);
        if (kk & 1) v1 = fmaf(lik, x[kk], v1);
        else v0 = fmaf(lik, x[kk], v0);
      }
      x[i] = (i > r) ? -(v0 + v1) * rinv : (i == r ? rinv : 0.0f);   // X(i, r), X = L^-1
    }
    float* Rib = Rinv + (size_t)b * LPB * LPB;
#pragma unroll
    for (int i = 0; i < LPB; ++i) Rib[r * LPB + i] = x[i];   // R^-1(r, i) = X(i, r)
  }
}

// rows x 32 floats into columns col0 .. col0 + 31 of dst (ldd and col0 multiples of 4):
// 16-byte elements, four loads in flight per thread
__global__ void copy_block_kernel(const float* __restrict__ src, int64_t rows, float* __restrict__ dst,
                                  int ldd, int col0) {
  const int64_t n4 = rows * (LPB / 4);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const float4* s4 = reinterpret_cast<const float4*>(src);
  auto put = [&](int64_t e, float4 v) {
    const int64_t r = e >> 3;
    *reinterpret_cast<float4*>(dst + r * ldd + col0 + 4 * (int)(e & 7)) = v;
  };
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e + 3 * stride < n4; e += 4 * stride) {
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = s4[e + u * stride];
#pragma unroll
    for (int u = 0; u < 4; ++u) put(e + u * stride, v[u]);
  }
  for (; e < n4; e += stride) put(e, s4[e]);
}

// x -> three bfloat16 planes h = bf16(x), m = bf16(x - h), t = bf16(x - h - m) (x to 24
// significant bits), planes [3][rows][kr], for the tensor-core form of dL/dA.
// (n a multiple of 4: four elements per step, 16-byte loads and 8-byte stores, two steps'
// loads in flight per thread)
__global__ void bwd_split_kernel(const float* __restrict__ x, int64_t n, __nv_bfloat16* __restrict__ planes) {
  const int64_t n4 = n / 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const float4* x4 = reinterpret_cast<const float4*>(x);
  auto put = [&](int64_t e, float4 v4) {
    const float v[4] = {v4.x, v4.y, v4.z, v4.w};
    __nv_bfloat16 h[4], mm[4], t[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      h[i] = __float2bfloat16_rn(v[i]);
      const float r1 = v[i] - __bfloat162float(h[i]);
      mm[i] = __float2bfloat16_rn(r1);
      t[i] = __float2bfloat16_rn(r1 - __bfloat162float(mm[i]));
    }
    auto st4 = [&](__nv_bfloat16* d, const __nv_bfloat16 (&q)[4]) {
      __nv_bfloat162 lo, hi;
      lo.x = q[0]; lo.y = q[1]; hi.x = q[2]; hi.y = q[3];
      uint2 w;
      w.x = *reinterpret_cast<const uint32_t*>(&lo);
      w.y = *reinterpret_cast<const uint32_t*>(&hi);
      *reinterpret_cast<uint2*>(d + 4 * e) = w;
    };
    st4(planes, h);
    st4(planes + n, mm);
    st4(planes + 2 * n, t);
  };
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e + stride < n4; e += 2 * stride) {
    const float4 a = x4[e], b = x4[e + stride];
    put(e, a);
    put(e + stride, b);
  }
  for (; e < n4; e += stride) put(e, x4[e]);
}

// dL/dA on the tensor cores: gA_b = 2 A_b + L_b R_b^T for 128 x 128 tiles (units: matrix,
// row tile, column tile; dealt round-robin to persistent CTAs).  The MMA forms the tile
// transposed, D = R L^T (tensor-memory lane = column of dL/dA, tensor-memory column = row),
// so that a warp holds 32 adjacent columns of one row in its 32 lanes: A is read and dL/dA
// written in coalesced rows straight from the accumulator.  L and R come as three bfloat16
// planes each; per k16 step six products (t h, h t, m m, m h, h m, h h, the small ones
// first) accumulate in float32, which carries L R^T to about 2^-22 of |L| |R|.  Warp 0
// loads the six 128 x 64 plane tiles of a k chunk by TMA (two stages of 96 KB) and the
// unit's tile of A (32 KB, after the previous unit's epilogue has read it), warp 1 issues
// the MMAs into a double-buffered accumulator, warps 2-5 write 2 A + D^T.
constexpr int kFT = 128;                                     // tile rows and columns
constexpr int kFinalThreads = 192;
constexpr uint32_t kPlaneTile = (uint32_t)kFT * 64 * 2;      // 128 rows x 64 k, bf16
constexpr uint32_t kFinalStage = 6 * kPlaneTile;             // 96 KB
constexpr int kFinalStages = 2;
constexpr uint32_t kATile = (uint32_t)kFT * kFT * 2;         // 32 KB: two 64-column boxes
constexpr size_t kFinalSmem = (size_t)kFinalStages * kFinalStage + kATile + 1024;

__global__ void __launch_bounds__(kFinalThreads, 1) bwd_final_tc_kernel(
    const __grid_constant__ CUtensorMap map_l, const __grid_constant__ CUtensorMap map_r,
    const CUtensorMap* __restrict__ maps_a, const int4* __restrict__ units, int nunits, int64_t sum_m,
    int64_t sum_n, int kr, float* const* __restrict__ gA, const int64_t* __restrict__ m,
    const int64_t* __restrict__ n, const int64_t* __restrict__ roff_m, const int64_t* __restrict__ roff_n,
    uint32_t* status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar_full[kFinalStages], bar_empty[kFinalStages], bar_acc_full[2], bar_acc_empty[2];
  __shared__ uint64_t bar_a_full, bar_a_empty;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint8_t* sA = smem + kFinalStages * kFinalStage;
  constexpr uint32_t acc_cols = kFT, tmem_cols = 2 * kFT;
  const int kc = kr / 64;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kFinalStages; ++s) {
      mbar_init(&bar_full[s], 1);
      mbar_init(&bar_empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&bar_acc_full[a], 1);
      mbar_init(&bar_acc_empty[a], 4);
    }
    mbar_init(&bar_a_full, 1);
    mbar_init(&bar_a_empty, 4);
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
      int j = 0;
      int a_loads = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x, ++j) {
        const int4 un = units[u];
        const int yl = (int)(roff_m[un.x] + (int64_t)un.y * kFT);
        const int yr = (int)(roff_n[un.x] + (int64_t)un.z * kFT);
        for (int kk = 0; kk < kc; ++kk, ++i) {
          const int s = (int)(i % kFinalStages);
          const uint32_t ph = (uint32_t)((i / kFinalStages) & 1);
          if (!mbar_wait(&bar_empty[s], ph ^ 1u, abort_flag, status)) { ok = false; break; }
          uint8_t* sa = smem + (size_t)s * kFinalStage;
          mbar_expect_tx(&bar_full[s], kFinalStage);
#pragma unroll
          for (int p = 0; p < 3; ++p) {   // MMA A operand: R (columns of dL/dA); B operand: L
            tma_load_2d(sa + p * kPlaneTile, &map_r, &bar_full[s], kk * 64, (int)(p * sum_n) + yr);
            tma_load_2d(sa + (3 + p) * kPlaneTile, &map_l, &bar_full[s], kk * 64, (int)(p * sum_m) + yl);
          }
        }
        if (!ok) break;
        // the tile of A once the previous unit's epilogue is done with the buffer
        if (!mbar_wait(&bar_a_empty, ((uint32_t)j & 1u) ^ 1u, abort_flag, status)) break;
        const CUtensorMap* ma = maps_a + un.x;
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                         reinterpret_cast<uint64_t>(ma))
                     : "memory");
        mbar_expect_tx(&bar_a_full, kATile);
        tma_load_2d(sA, ma, &bar_a_full, un.z * kFT, un.y * kFT);
        tma_load_2d(sA + kATile / 2, ma, &bar_a_full, un.z * kFT + 64, un.y * kFT);
        ++a_loads;
      }
      // let the copies in flight land before the CTA can exit
      const int64_t issued = i;
      for (int64_t t = (issued > kFinalStages ? issued - kFinalStages : 0); t < issued; ++t) {
        const int s = (int)(t % kFinalStages);
        const uint32_t ph = (uint32_t)((t / kFinalStages) & 1);
        for (uint32_t w = 0; w < kSpinLimit && !mbar_try_wait(&bar_full[s], ph); ++w) __nanosleep(64);
      }
      if (a_loads > 0) {
        const uint32_t ph = (uint32_t)((a_loads - 1) & 1);
        for (uint32_t w = 0; w < kSpinLimit && !mbar_try_wait(&bar_a_full, ph); ++w) __nanosleep(64);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = instr_desc(kFT, 0);
      // (R plane, L plane): the smallest products first
      constexpr int pa[6] = {2, 0, 1, 1, 0, 0};
      constexpr int pb[6] = {0, 2, 1, 0, 1, 0};
      int64_t i = 0;
      int j = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x, ++j) {
        const int ab = j & 1;
        if (!mbar_wait(&bar_acc_empty[ab], ((uint32_t)(j >> 1) & 1u) ^ 1u, abort_flag, status)) break;
        tc_fence_after();
        const uint32_t dst = tmem + ab * acc_cols;
        for (int kk = 0; kk < kc; ++kk, ++i) {
          const int s = (int)(i % kFinalStages);
          const uint32_t ph = (uint32_t)((i / kFinalStages) & 1);
          if (!mbar_wait(&bar_full[s], ph, abort_flag, status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + (size_t)s * kFinalStage);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
#pragma unroll
            for (int t = 0; t < 6; ++t) {
              const uint64_t adesc = smem_desc(sa + pa[t] * kPlaneTile + q * 32, 16, 1024);
              const uint64_t bdesc = smem_desc(sa + (3 + pb[t]) * kPlaneTile + q * 32, 16, 1024);
              mma_bf16(dst, adesc, bdesc, idesc, (kk == 0 && q == 0 && t == 0) ? 0u : 1u);
            }
          }
          mma_commit(&bar_empty[s]);
        }
        if (ok) mma_commit(&bar_acc_full[ab]);
      }
    }
  } else {
    const int quad = warp & 3;            // the tensor-memory lane quarter this warp may read
    const int cl = quad * 32 + lane;      // column of the tile
    // the swizzled position of column cl in a 128-byte row of the A tile (two 64-column boxes)
    const uint32_t box_off = (uint32_t)(cl >> 6) * (kATile / 2);
    const int chunk16 = (cl & 63) >> 3, within = (cl & 7) * 2;
    int j = 0;
    for (int u = blockIdx.x; u < nunits; u += gridDim.x, ++j) {
      const int4 un = units[u];
      const int ab = j & 1;
      bool ok = mbar_wait(&bar_acc_full[ab], (uint32_t)(j >> 1) & 1u, abort_flag, status);
      ok = ok && mbar_wait(&bar_a_full, (uint32_t)j & 1u, abort_flag, status);
      ok = __all_sync(0xffffffffu, ok);
      tc_fence_after();
      if (ok) {
        const int b = un.x;
        const int64_t mb = m[b], nb = n[b];
        const int64_t rbase = (int64_t)un.y * kFT, c = (int64_t)un.z * kFT + cl;
        float* __restrict__ G = gA[b];
        for (int c0 = 0; c0 < kFT && rbase + c0 < mb; c0 += 32) {
          float v[32];
          tmem_ld32(tmem + ab * acc_cols + c0 + ((uint32_t)(quad * 32) << 16), v);
          if (c < nb) {
#pragma unroll
            for (int t = 0; t < 32; ++t) {
              const int rl = c0 + t;
              const int64_t r = rbase + rl;
              const uint32_t off = box_off + (uint32_t)rl * 128 + (uint32_t)((chunk16 ^ (rl & 7)) << 4) + within;
              const float a = __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(sA + off));
              if (r < mb) G[r * nb + c] = fmaf(2.0f, a, v[t]);
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&bar_a_empty);
        mbar_arrive(&bar_acc_empty[ab]);
      }
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

}  // namespace

cudaError_t launch_bwd_gq(const float* P, const float* Q, const int64_t* roff, const int2* units, int nunits,
                          const float* ut, const float* sig, int k, float* gq, float* ublk, int ldu,
                          cudaStream_t st) {
  if (nunits <= 0) return cudaSuccess;
  bwd_gq_kernel<<<nunits, kUT, 0, st>>>(P, Q, roff, units, ut, sig, k, gq, ublk, ldu);
  return cudaGetLastError();
}

cudaError_t launch_bwd_qr_small(const float* Q, const float* gQ, const int64_t* roff, const int2* units,
                                int nunits, const int* ustart, int nb, int l, const float* R, float* part,
                                float* N, float* Rinv, cudaStream_t st) {
  if (nunits <= 0) return cudaSuccess;
  bwd_cross_kernel<<<nunits, 256, 0, st>>>(gQ, Q, roff, units, part);
  bwd_qr_small_kernel<<<nb, 128, 0, st>>>(part, ustart, l, R, N, Rinv);
  return cudaGetLastError();
}

cudaError_t launch_bwd_qr_apply(const float* Q, const float* gQ, const int64_t* roff, const int2* units,
                                int nunits, const float* N, const float* Rinv, float* gY, cudaStream_t st) {
  if (nunits <= 0) return cudaSuccess;
  bwd_qr_apply_kernel<<<nunits, kUT, 0, st>>>(Q, gQ, roff, units, N, Rinv, gY);
  return cudaGetLastError();
}

cudaError_t launch_copy_block(const float* src, int64_t rows, float* dst, int ldd, int col0,
                              cudaStream_t st) {
  if (ldd % 4 || col0 % 4 || ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15))
    return cudaErrorInvalidValue;
  const int64_t n = rows * (LPB / 4);
  const int64_t blocks = cdiv(n, 256);
  copy_block_kernel<<<(unsigned)(blocks < 16 * kNumSMs ? blocks : 16 * kNumSMs), 256, 0, st>>>(
      src, rows, dst, ldd, col0);
  return cudaGetLastError();
}

cudaError_t launch_bwd_split(const float* x, int64_t n, __nv_bfloat16* planes, cudaStream_t st) {
  if (n % 4 || ((reinterpret_cast<uintptr_t>(x) & 15) | (reinterpret_cast<uintptr_t>(planes) & 7)))
    return cudaErrorInvalidValue;
  const int64_t blocks = cdiv(n / 4, 256);
  bwd_split_kernel<<<(unsigned)(blocks < 16 * kNumSMs ? blocks : 16 * kNumSMs), 256, 0, st>>>(x, n, planes);
  return cudaGetLastError();
}

cudaError_t prepare_batched_bwd() {
  return cudaFuncSetAttribute(bwd_final_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kFinalSmem);
}

int bwd_final_tile() { return kFT; }

cudaError_t launch_bwd_final(const void* map_l, const void* map_r, const void* maps_a, const int4* units,
                             int nunits, int64_t sum_m, int64_t sum_n, int kr, float* const* gA,
                             const int64_t* m, const int64_t* n, const int64_t* roff_m, const int64_t* roff_n,
                             int grid, uint32_t* status, cudaStream_t st) {
  if (nunits <= 0) return cudaSuccess;
  if (kr % 64 || kr <= 0 || 3 * (sum_m > sum_n ? sum_m : sum_n) >= ((int64_t)1 << 31))
    return cudaErrorInvalidValue;
  if (grid > nunits) grid = nunits;
  bwd_final_tc_kernel<<<grid, kFinalThreads, kFinalSmem, st>>>(
      *static_cast<const CUtensorMap*>(map_l), *static_cast<const CUtensorMap*>(map_r),
      static_cast<const CUtensorMap*>(maps_a), units, nunits, sum_m, sum_n, kr, gA, m, n, roff_m, roff_n,
      status);
  return cudaGetLastError();
}

}  // namespace rsvd
