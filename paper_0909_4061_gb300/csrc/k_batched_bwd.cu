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
#include "batched_rows.cuh"
#include "kernels_batched.cuh"
#include "tc_ptx.cuh"

namespace rsvd {
namespace {

using namespace tcx;

constexpr int LPB = 32;

static_assert(LPB == kTileWidth, "the basis rows are the row tiles of batched_rows.cuh");

// rows of the Cholesky-QR unit u = (matrix, 128-row tile)
__device__ __forceinline__ void unit_rows(const int64_t* __restrict__ roff, int2 u, int64_t* row0, int* nr) {
  *row0 = roff[u.x] + (int64_t)u.y * kTileRows;
  *nr = (int)min((int64_t)kTileRows, roff[u.x + 1] - *row0);
}

// The row kernels below take a thread per row of a Cholesky-QR unit (kTileRows threads):
// the unit's rows are staged by coalesced loads (batched_rows.cuh), a thread holds its row's
// first 4 L4 entries in registers (L4 = ceil(l / 4): the basis columns beyond l are zero),
// the per-matrix factors sit in shared memory and are read as float4 broadcasts, the sums
// run in index order, and the results leave through the staged tile by coalesced stores.

// t_c = P[r][c] (1 - 2 s_c) + 2 s_c^2 u_c with u = Q[r] Ut; gQ[r][i] = sum_{c<k} t_c Ut[i][c];
// ublk[r][c] = u_c (1 - 2 s_c) for c < k, zero beyond (the first left factor U (I - 2S)).
template <int L4>
__global__ void __launch_bounds__(kTileRows) bwd_gq_kernel(const float* __restrict__ P, const float* __restrict__ Q,
                                                           const int64_t* __restrict__ roff,
                                                           const int2* __restrict__ units,
                                                           const float* __restrict__ ut, const float* __restrict__ sig,
                                                           int k, float* __restrict__ gq, float* __restrict__ ublk,
                                                           int ldu) {
  constexpr int LC = 4 * L4;
  __shared__ __align__(16) float qs[kTileRows * kRowStride];
  __shared__ __align__(16) float ps[kTileRows * kRowStride];
  __shared__ __align__(16) float Us[LC][LPB];     // rows 0 .. LC - 1 of Ut
  __shared__ __align__(16) float cf[2][LPB];      // 1 - 2 s_c and 2 s_c^2, zero for c >= k
  const int2 u = units[blockIdx.x];
  int64_t row0;
  int nr;
  unit_rows(roff, u, &row0, &nr);
  const int t = threadIdx.x;
  stage_tile<L4>(Q, row0, nr, qs);
  stage_tile<L4>(P, row0, nr, ps);
  for (int e = t; e < LC * LPB; e += kTileRows) Us[e / LPB][e % LPB] = ut[(size_t)u.x * LPB * LPB + e];
  if (t < LPB) {
    const float s = t < k ? sig[(size_t)u.x * LPB + t] : 0.0f;
    cf[0][t] = t < k ? 1.0f - 2.0f * s : 0.0f;
    cf[1][t] = t < k ? 2.0f * s * s : 0.0f;
  }
  __syncthreads();
  float y[LC], pr[LC];
  load_row<L4>(qs, t, y);
  load_row<L4>(ps, t, pr);
  const int k4 = (k + 3) >> 2;
  float tv[LC];
  float4 ub[L4];
#pragma unroll
  for (int c4 = 0; c4 < L4; ++c4) {
    float4 uc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (c4 < k4) {
#pragma unroll
      for (int j = 0; j < LC; ++j) {
        const float4 w = *reinterpret_cast<const float4*>(&Us[j][4 * c4]);
        uc.x = fmaf(y[j], w.x, uc.x);
        uc.y = fmaf(y[j], w.y, uc.y);
        uc.z = fmaf(y[j], w.z, uc.z);
        uc.w = fmaf(y[j], w.w, uc.w);
      }
    }
    const float4 c1 = *reinterpret_cast<const float4*>(&cf[0][4 * c4]);
    const float4 c2 = *reinterpret_cast<const float4*>(&cf[1][4 * c4]);
    tv[4 * c4] = fmaf(pr[4 * c4], c1.x, c2.x * uc.x);
    tv[4 * c4 + 1] = fmaf(pr[4 * c4 + 1], c1.y, c2.y * uc.y);
    tv[4 * c4 + 2] = fmaf(pr[4 * c4 + 2], c1.z, c2.z * uc.z);
    tv[4 * c4 + 3] = fmaf(pr[4 * c4 + 3], c1.w, c2.w * uc.w);
    ub[c4] = make_float4(uc.x * c1.x, uc.y * c1.y, uc.z * c1.z, uc.w * c1.w);
  }
  // row t of both tiles is read by this thread alone (its rows are in registers)
#pragma unroll
  for (int i4 = 0; i4 < L4; ++i4) {
    float g[4];
#pragma unroll
    for (int ii = 0; ii < 4; ++ii) {
      const int i = 4 * i4 + ii;
      float a = 0.0f;
#pragma unroll
      for (int c4 = 0; c4 < L4; ++c4) {
        if (c4 < k4) {
          const float4 w = *reinterpret_cast<const float4*>(&Us[i][4 * c4]);
          a = fmaf(tv[4 * c4], w.x, a);
          a = fmaf(tv[4 * c4 + 1], w.y, a);
          a = fmaf(tv[4 * c4 + 2], w.z, a);
          a = fmaf(tv[4 * c4 + 3], w.w, a);
        }
      }
      g[ii] = a;
    }
    *reinterpret_cast<float4*>(qs + t * kRowStride + 4 * i4) = make_float4(g[0], g[1], g[2], g[3]);
    *reinterpret_cast<float4*>(ps + t * kRowStride + 4 * i4) = ub[i4];
  }
  __syncthreads();
  store_tile<L4>(qs, nr, gq, row0, LPB);
  store_tile<L4>(ps, nr, ublk, row0, ldu);
}

// gY = (gQ + Q N) R^-T per row: w_j = gQ[r][j] + sum_t Q[r][t] N[t][j], then
// gY[r][i] = sum_{j >= i} w_j Rinv[i][j] (R^-1 is upper triangular).
template <int L4>
__global__ void __launch_bounds__(kTileRows) bwd_qr_apply_kernel(const float* __restrict__ Q,
                                                                 const float* __restrict__ gQ,
                                                                 const int64_t* __restrict__ roff,
                                                                 const int2* __restrict__ units,
                                                                 const float* __restrict__ N,
                                                                 const float* __restrict__ Rinv,
                                                                 float* __restrict__ gY) {
  constexpr int LC = 4 * L4;
  __shared__ __align__(16) float qs[kTileRows * kRowStride];
  __shared__ __align__(16) float gs[kTileRows * kRowStride];
  __shared__ __align__(16) float Ns[LC][LPB];
  __shared__ __align__(16) float Rs[LC][LPB];
  const int2 u = units[blockIdx.x];
  int64_t row0;
  int nr;
  unit_rows(roff, u, &row0, &nr);
  const int t = threadIdx.x;
  stage_tile<L4>(Q, row0, nr, qs);
  stage_tile<L4>(gQ, row0, nr, gs);
  for (int e = t; e < LC * LPB; e += kTileRows) {
    Ns[e / LPB][e % LPB] = N[(size_t)u.x * LPB * LPB + e];
    Rs[e / LPB][e % LPB] = Rinv[(size_t)u.x * LPB * LPB + e];
  }
  __syncthreads();
  float y[LC], g[LC];
  load_row<L4>(qs, t, y);
  load_row<L4>(gs, t, g);
  float w[LC];
#pragma unroll
  for (int j4 = 0; j4 < L4; ++j4) {
    float4 acc = make_float4(g[4 * j4], g[4 * j4 + 1], g[4 * j4 + 2], g[4 * j4 + 3]);
#pragma unroll
    for (int s = 0; s < LC; ++s) {
      const float4 n4 = *reinterpret_cast<const float4*>(&Ns[s][4 * j4]);
      acc.x = fmaf(y[s], n4.x, acc.x);
      acc.y = fmaf(y[s], n4.y, acc.y);
      acc.z = fmaf(y[s], n4.z, acc.z);
      acc.w = fmaf(y[s], n4.w, acc.w);
    }
    w[4 * j4] = acc.x; w[4 * j4 + 1] = acc.y; w[4 * j4 + 2] = acc.z; w[4 * j4 + 3] = acc.w;
  }
#pragma unroll
  for (int i4 = 0; i4 < L4; ++i4) {
    float o[4];
#pragma unroll
    for (int ii = 0; ii < 4; ++ii) {
      const int i = 4 * i4 + ii;
      float a = 0.0f;
#pragma unroll
      for (int j4 = i4; j4 < L4; ++j4) {
        const float4 r4 = *reinterpret_cast<const float4*>(&Rs[i][4 * j4]);
        a = fmaf(w[4 * j4], r4.x, a);
        a = fmaf(w[4 * j4 + 1], r4.y, a);
        a = fmaf(w[4 * j4 + 2], r4.z, a);
        a = fmaf(w[4 * j4 + 3], r4.w, a);
      }
      o[ii] = a;
    }
    *reinterpret_cast<float4*>(qs + t * kRowStride + 4 * i4) = make_float4(o[0], o[1], o[2], o[3]);
  }
  __syncthreads();
  store_tile<L4>(qs, nr, gY, row0, LPB);
}

// C_u = sum over the rows of a Cholesky-QR unit (matrix b, 128-row tile) of gQ[r][i] Q[r][j]
// for i, j < 4 L4 (zero beyond): the partial of gQ^T Q.  The L4 x L4 tiles of 4 x 4 each
// have one thread in each of NG = 128 / L4^2 row groups (two float4 reads per 16 FMAs);
// the groups are summed in a fixed order through shared memory.
template <int L4>
__global__ void __launch_bounds__(kTileRows) bwd_cross_kernel(const float* __restrict__ gQ, const float* __restrict__ Q,
                                                              const int64_t* __restrict__ roff,
                                                              const int2* __restrict__ units, float* __restrict__ part) {
  constexpr int NTILE = L4 * L4;
  constexpr int NG = kTileRows / NTILE;
  __shared__ __align__(16) float gs[kTileRows * kRowStride];
  __shared__ __align__(16) float qs[kTileRows * kRowStride];
  __shared__ __align__(16) float gp[NG * NTILE * 16];
  const int2 u = units[blockIdx.x];
  int64_t row0;
  int nr;
  unit_rows(roff, u, &row0, &nr);
  stage_tile<L4>(gQ, row0, nr, gs);
  stage_tile<L4>(Q, row0, nr, qs);
  __syncthreads();
  const int grp = threadIdx.x / NTILE, tt = threadIdx.x - grp * NTILE;
  if (grp < NG) {
    const int bi = 4 * (tt / L4), bj = 4 * (tt % L4);
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
#pragma unroll 4
    for (int rr = grp; rr < nr; rr += NG) {
      const float4 x = *reinterpret_cast<const float4*>(gs + rr * kRowStride + bi);
      const float4 y = *reinterpret_cast<const float4*>(qs + rr * kRowStride + bj);
      const float xv[4] = {x.x, x.y, x.z, x.w}, yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xv[i], yv[j], acc[i][j]);
    }
    float* d = gp + (grp * NTILE + tt) * 16;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      *reinterpret_cast<float4*>(d + 4 * i) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
  }
  __syncthreads();
  float* pu = part + (size_t)blockIdx.x * LPB * LPB;
  for (int e = threadIdx.x; e < LPB * LPB; e += kTileRows) {
    const int i = e >> 5, j = e & 31, ti = i >> 2, tj = j >> 2;
    float v = 0.0f;
    if (ti < L4 && tj < L4) {
      const int off = (ti * L4 + tj) * 16 + (i & 3) * 4 + (j & 3);
#pragma unroll
      for (int g = 0; g < NG; ++g) v += gp[g * NTILE * 16 + off];
    }
    pu[e] = v;
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

#define RSVD_L4_SWITCH(l, CASE)                                                          \
  switch (((l) + 3) / 4) {                                                               \
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)                      \
    default: return cudaErrorInvalidValue;                                               \
  }

cudaError_t launch_bwd_gq(const float* P, const float* Q, const int64_t* roff, const int2* units, int nunits,
                          int l, const float* ut, const float* sig, int k, float* gq, float* ublk, int ldu,
                          cudaStream_t st) {
  if (nunits <= 0) return cudaSuccess;
  if (k > l || ldu % 4 || (reinterpret_cast<uintptr_t>(ublk) & 15)) return cudaErrorInvalidValue;
#define RSVD_GQ(L4)                                                                                   \
  case L4:                                                                                           \
    bwd_gq_kernel<L4><<<nunits, kTileRows, 0, st>>>(P, Q, roff, units, ut, sig, k, gq, ublk, ldu);   \
    break;
  RSVD_L4_SWITCH(l, RSVD_GQ)
#undef RSVD_GQ
  return cudaGetLastError();
}

cudaError_t launch_bwd_qr_small(const float* Q, const float* gQ, const int64_t* roff, const int2* units,
                                int nunits, const int* ustart, int nb, int l, const float* R, float* part,
                                float* N, float* Rinv, cudaStream_t st) {
  if (nunits <= 0) return cudaSuccess;
#define RSVD_CROSS(L4)                                                                 \
  case L4:                                                                            \
    bwd_cross_kernel<L4><<<nunits, kTileRows, 0, st>>>(gQ, Q, roff, units, part);     \
    break;
  RSVD_L4_SWITCH(l, RSVD_CROSS)
#undef RSVD_CROSS
  bwd_qr_small_kernel<<<nb, 128, 0, st>>>(part, ustart, l, R, N, Rinv);
  return cudaGetLastError();
}

cudaError_t launch_bwd_qr_apply(const float* Q, const float* gQ, const int64_t* roff, const int2* units,
                                int nunits, int l, const float* N, const float* Rinv, float* gY, cudaStream_t st) {
  if (nunits <= 0) return cudaSuccess;
#define RSVD_QRA(L4)                                                                        \
  case L4:                                                                                 \
    bwd_qr_apply_kernel<L4><<<nunits, kTileRows, 0, st>>>(Q, gQ, roff, units, N, Rinv, gY); \
    break;
  RSVD_L4_SWITCH(l, RSVD_QRA)
#undef RSVD_QRA
  return cudaGetLastError();
}
#undef RSVD_L4_SWITCH

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
