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
#include "common.cuh"
#include "kernels_batched.cuh"

namespace rsvd {
namespace {

constexpr int LPB = 32;

// one CTA per matrix (Ut, sigma in shared memory), one warp per row: lane c forms
// t_c = P[r][c] (1 - 2 s_c) + 2 s_c^2 u_c with u_c = (Q Ut)[r][c]; lane i then
// gQ[r][i] = sum_{c<k} t_c Ut[i][c]
__global__ void __launch_bounds__(256) bwd_gq_kernel(const float* __restrict__ P,
                                                     const float* __restrict__ Q,
                                                     const int64_t* __restrict__ roff,
                                                     const float* __restrict__ ut,
                                                     const float* __restrict__ sig, int k,
                                                     float* __restrict__ gq, float* __restrict__ ublk,
                                                     int ldu) {
  __shared__ float Us[LPB][LPB + 1];
  __shared__ float ss[LPB];
  const int b = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < LPB * LPB; e += blockDim.x) Us[e / LPB][e % LPB] = ut[(size_t)b * LPB * LPB + e];
  if (threadIdx.x < LPB) ss[threadIdx.x] = threadIdx.x < k ? sig[(size_t)b * LPB + threadIdx.x] : 0.0f;
  __syncthreads();
  const float s = ss[lane];
  const float c1 = 1.0f - 2.0f * s, c2 = 2.0f * s * s;
  for (int64_t r = roff[b] + warp; r < roff[b + 1]; r += blockDim.x >> 5) {
    const float qv = Q[r * LPB + lane];
    float u0 = 0.0f, u1 = 0.0f;
#pragma unroll
    for (int j = 0; j < LPB; j += 2) {
      u0 = fmaf(__shfl_sync(0xffffffffu, qv, j), Us[j][lane], u0);
      u1 = fmaf(__shfl_sync(0xffffffffu, qv, j + 1), Us[j + 1][lane], u1);
    }
    const float u = u0 + u1;
    const float t = lane < k ? fmaf(P[r * LPB + lane], c1, c2 * u) : 0.0f;
    ublk[r * ldu + lane] = lane < k ? u * c1 : 0.0f;
    float g0 = 0.0f, g1 = 0.0f;
#pragma unroll
    for (int c = 0; c < LPB; c += 2) {   // t_c = 0 for c >= k
      g0 = fmaf(__shfl_sync(0xffffffffu, t, c), Us[lane][c], g0);
      g1 = fmaf(__shfl_sync(0xffffffffu, t, c + 1), Us[lane][c + 1], g1);
    }
    gq[r * LPB + lane] = g0 + g1;
  }
}

// one CTA per matrix: C = gQ^T Q (rows staged in shared memory), N = copyltu(-C);
// Rinv = R^-1 from R^T = L lower: warp 0, lane r holds row r of L, X = L^-1 by columns.
constexpr int kSmallThreads = 256;
constexpr int kRows = 64;

__global__ void __launch_bounds__(kSmallThreads) bwd_qr_small_kernel(
    const float* __restrict__ Q, const float* __restrict__ gQ, const int64_t* __restrict__ roff, int l,
    const float* __restrict__ R, float* __restrict__ N, float* __restrict__ Rinv) {
  __shared__ float qs[kRows][LPB];
  __shared__ float gs[kRows][LPB];
  __shared__ float C[LPB][LPB + 1];
  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = roff[b], rows = roff[b + 1] - r0;
  const int gi = 4 * warp, gj = lane;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int64_t c0 = 0; c0 < rows; c0 += kRows) {
    const int nr = (int)min((int64_t)kRows, rows - c0);
    __syncthreads();
    for (int e = tid; e < kRows * LPB; e += kSmallThreads) {
      const int rr = e / LPB, cc = e % LPB;
      qs[rr][cc] = rr < nr ? Q[(r0 + c0 + rr) * LPB + cc] : 0.0f;
      gs[rr][cc] = rr < nr ? gQ[(r0 + c0 + rr) * LPB + cc] : 0.0f;
    }
    __syncthreads();
    for (int rr = 0; rr < nr; ++rr) {
      const float qj = qs[rr][gj];
#pragma unroll
      for (int a = 0; a < 4; ++a) acc[a] = fmaf(gs[rr][gi + a], qj, acc[a]);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) C[gi + a][gj] = acc[a];   // C(i, j) = sum_r gQ[r][i] Q[r][j]
  __syncthreads();
  float* Nb = N + (size_t)b * LPB * LPB;
  for (int e = tid; e < LPB * LPB; e += kSmallThreads) {
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

// one CTA per matrix (N, R^-1 in shared memory), one warp per row: lane j:
// w_j = gQ[r][j] + sum_t Q[r][t] N[t][j]; lane i: gY[r][i] = sum_j w_j Rinv[i][j] (gY = w R^-T)
__global__ void __launch_bounds__(256) bwd_qr_apply_kernel(const float* __restrict__ Q,
                                                           const float* __restrict__ gQ,
                                                           const int64_t* __restrict__ roff,
                                                           const float* __restrict__ N,
                                                           const float* __restrict__ Rinv,
                                                           float* __restrict__ gY) {
  __shared__ float Ns[LPB][LPB + 1];
  __shared__ float Rs[LPB][LPB + 1];
  const int b = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < LPB * LPB; e += blockDim.x) {
    Ns[e / LPB][e % LPB] = N[(size_t)b * LPB * LPB + e];
    Rs[e / LPB][e % LPB] = Rinv[(size_t)b * LPB * LPB + e];
  }
  __syncthreads();
  for (int64_t r = roff[b] + warp; r < roff[b + 1]; r += blockDim.x >> 5) {
    const float qv = Q[r * LPB + lane];
    float w0 = gQ[r * LPB + lane], w1 = 0.0f;
#pragma unroll
    for (int t = 0; t < LPB; t += 2) {
      w0 = fmaf(__shfl_sync(0xffffffffu, qv, t), Ns[t][lane], w0);
      w1 = fmaf(__shfl_sync(0xffffffffu, qv, t + 1), Ns[t + 1][lane], w1);
    }
    const float w = w0 + w1;
    float g0 = 0.0f, g1 = 0.0f;
#pragma unroll
    for (int j = 0; j < LPB; j += 2) {
      g0 = fmaf(__shfl_sync(0xffffffffu, w, j), Rs[lane][j], g0);
      g1 = fmaf(__shfl_sync(0xffffffffu, w, j + 1), Rs[lane][j + 1], g1);
    }
    gY[r * LPB + lane] = g0 + g1;
  }
}

__global__ void copy_block_kernel(const float* __restrict__ src, int64_t rows, float* __restrict__ dst,
                                  int ldd, int col0) {
  const int64_t n = rows * LPB;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / LPB;
    const int c = (int)(e - r * LPB);
    dst[r * ldd + col0 + c] = src[e];
  }
}

// gA_b[r][c] = 2 A_b[r][c] + sum_t L[rm_b + r][t] R[rn_b + c][t] on a 64 x 64 tile per CTA;
// 256 threads, 4 x 4 outputs each, K in chunks of 32 through shared memory
constexpr int FT = 64;

__global__ void __launch_bounds__(256) bwd_final_kernel(
    const int4* __restrict__ units, const void* const* __restrict__ A, const int64_t* __restrict__ lda,
    float* const* __restrict__ gA, const int64_t* __restrict__ m, const int64_t* __restrict__ n,
    const int64_t* __restrict__ roff_m, const int64_t* __restrict__ roff_n, const float* __restrict__ L,
    const float* __restrict__ R, int kr) {
  __shared__ float Ls[32][FT + 4];   // Ls[t][row]
  __shared__ float Rs[32][FT + 4];   // Rs[t][col]
  const int4 u = units[blockIdx.x];
  const int b = u.x;
  const int64_t mb = m[b], nbc = n[b];
  const int64_t rt0 = (int64_t)u.y * FT, ct0 = (int64_t)u.z * FT;
  const float* Lb = L + roff_m[b] * kr;
  const float* Rb = R + roff_n[b] * kr;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4] = {};
  for (int t0 = 0; t0 < kr; t0 += 32) {
    __syncthreads();
    for (int e = tid; e < FT * 32; e += 256) {
      const int rr = e >> 5, t = e & 31;
      const int64_t gr = rt0 + rr, gc = ct0 + rr;
      Ls[t][rr] = gr < mb ? Lb[gr * kr + t0 + t] : 0.0f;
      Rs[t][rr] = gc < nbc ? Rb[gc * kr + t0 + t] : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int t = 0; t < 32; ++t) {
      const float4 lv = *reinterpret_cast<const float4*>(&Ls[t][ty * 4]);
      const float4 rv = *reinterpret_cast<const float4*>(&Rs[t][tx * 4]);
      const float la[4] = {lv.x, lv.y, lv.z, lv.w}, ra[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(la[i], ra[j], acc[i][j]);
    }
  }
  const __nv_bfloat16* Ab = static_cast<const __nv_bfloat16*>(A[b]);
  float* G = gA[b];
  const int64_t ld = lda[b];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t r = rt0 + ty * 4 + i;
    if (r >= mb) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t c = ct0 + tx * 4 + j;
      if (c < nbc) G[r * nbc + c] = fmaf(2.0f, __bfloat162float(Ab[r * ld + c]), acc[i][j]);
    }
  }
}

}  // namespace

cudaError_t launch_bwd_gq(const float* P, const float* Q, const int64_t* roff, int nb, int64_t total_rows,
                          const float* ut, const float* sig, int k, float* gq, float* ublk, int ldu,
                          cudaStream_t st) {
  (void)total_rows;
  bwd_gq_kernel<<<nb, 256, 0, st>>>(P, Q, roff, ut, sig, k, gq, ublk, ldu);
  return cudaGetLastError();
}

cudaError_t launch_bwd_qr_small(const float* Q, const float* gQ, const int64_t* roff, int nb, int l,
                                const float* R, float* N, float* Rinv, cudaStream_t st) {
  bwd_qr_small_kernel<<<nb, kSmallThreads, 0, st>>>(Q, gQ, roff, l, R, N, Rinv);
  return cudaGetLastError();
}

cudaError_t launch_bwd_qr_apply(const float* Q, const float* gQ, const int64_t* roff, int nb,
                                int64_t total_rows, const float* N, const float* Rinv, float* gY,
                                cudaStream_t st) {
  (void)nb;
  (void)total_rows;
  bwd_qr_apply_kernel<<<nb, 256, 0, st>>>(Q, gQ, roff, N, Rinv, gY);
  return cudaGetLastError();
}

cudaError_t launch_copy_block(const float* src, int64_t rows, float* dst, int ldd, int col0,
                              cudaStream_t st) {
  const int64_t n = rows * LPB;
  const int64_t blocks = cdiv(n, 256);
  copy_block_kernel<<<(unsigned)(blocks < 16 * kNumSMs ? blocks : 16 * kNumSMs), 256, 0, st>>>(
      src, rows, dst, ldd, col0);
  return cudaGetLastError();
}

cudaError_t launch_bwd_final(const int4* units, int nunits, const void* const* A, const int64_t* lda,
                             float* const* gA, const int64_t* m, const int64_t* n,
                             const int64_t* roff_m, const int64_t* roff_n, const float* L,
                             const float* R, int kr, cudaStream_t st) {
  if (nunits <= 0) return cudaSuccess;
  bwd_final_kernel<<<nunits, 256, 0, st>>>(units, A, lda, gA, m, n, roff_m, roff_n, L, R, kr);
  return cudaGetLastError();
}

}  // namespace rsvd
