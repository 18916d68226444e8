// Kernels of the single-matrix backward pass (rsvd_svd_backward): the reverse of
// Algorithm 4.4 (Stage A) and Algorithm 5.1 (Stage B) with the test matrix held
// fixed.  The passes over A reuse the forward pass kernels; what is specific to the
// backward is here:
//   * small l x l steps: the SVD adjoint of B (F o (J - J^T) S + S F o (K - K^T) +
//     diag(gS), F_ij = 1 / (s_j^2 - s_i^2)), the antisymmetric part of a QR adjoint
//     (copyltu);
//   * row-wise steps on tall matrices: the cotangents of the reconstruction loss, column
//     scalings;
//   * the gradient itself, gA = alpha A + beta gA + L R^T, a tiled float32 GEMM whose
//     epilogue reads A (float32, bfloat16, or bfloat16 hi + lo) in the same tile.
#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {
namespace {

// ---- gA = alpha A + beta gA + L R^T --------------------------------------------------
// 128 x 128 tile of gA per CTA, 256 threads with an 8 x 8 register tile each (rows
// ty + 16 i, columns tx + 16 j), the K extent (columns of L and R) in slabs of 16 staged
// transposed in shared memory.
constexpr int LT = 128, LK = 16;

template <int ADT>   // 0: A float32, 1: bfloat16, 2: bfloat16 hi + lo (lo m * lda further)
__global__ void __launch_bounds__(256) lowrank_update_kernel(
    int64_t m, int64_t n, int kr, const float* __restrict__ L, int64_t ldl,
    const float* __restrict__ R, int64_t ldr, const void* __restrict__ A, int64_t lda, float alpha,
    float beta, float* __restrict__ G, int64_t ldg) {
  __shared__ float Ls[LK][LT + 4];
  __shared__ float Rs[LK][LT + 4];
  const int64_t r0 = (int64_t)blockIdx.y * LT, c0 = (int64_t)blockIdx.x * LT;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
  for (int t0 = 0; t0 < kr; t0 += LK) {
    __syncthreads();
    // 128 rows x 16 columns of L and of R: 8 elements per thread each
    for (int e = tid; e < LT * LK; e += 256) {
      const int rr = e / LK, t = e % LK;
      const int64_t gr = r0 + rr, gc = c0 + rr;
      Ls[t][rr] = (gr < m && t0 + t < kr) ? L[gr * ldl + t0 + t] : 0.0f;
      Rs[t][rr] = (gc < n && t0 + t < kr) ? R[gc * ldr + t0 + t] : 0.0f;
    }
    __syncthreads();
#pragma unroll 4
    for (int t = 0; t < LK; ++t) {
      float la[8], ra[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        la[i] = Ls[t][ty + 16 * i];
        ra[i] = Rs[t][tx + 16 * i];
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(la[i], ra[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t r = r0 + ty + 16 * i;
    if (r >= m) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t c = c0 + tx + 16 * j;
      if (c >= n) continue;
      float v = acc[i][j];
      if (alpha != 0.0f) {
        float a;
        if (ADT == 0) {
          a = static_cast<const float*>(A)[r * lda + c];
        } else {
          const __nv_bfloat16* ab = static_cast<const __nv_bfloat16*>(A);
          a = __bfloat162float(ab[r * lda + c]);
          if (ADT == 2) a += __bfloat162float(ab[(m + r) * lda + c]);
        }
        v = fmaf(alpha, a, v);
      }
      float* g = G + r * ldg + c;
      if (beta != 0.0f) v = fmaf(beta, *g, v);
      *g = v;
    }
  }
}

// ---- l x l steps (one CTA) -----------------------------------------------------------

// N = -copyltu(C): N_ij = -C_ij for i >= j, -C_ji above the diagonal (the QR adjoint's
// symmetric part, M = -gQ^T Q with its lower triangle mirrored).
__global__ void copyltu_neg_kernel(const float* __restrict__ C, int lp, float* __restrict__ N) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= lp * lp) return;
  const int i = e / lp, j = e % lp;
  N[e] = -(i >= j ? C[(int64_t)i * lp + j] : C[(int64_t)j * lp + i]);
}

// SVD adjoint of B = Ut S V_B^T (l x n, l <= n): with J = Ut^T gUt and K = V_B^T gV_B
// (only the first k columns of gUt, gV_B are nonzero) and F_ij = 1 / (s_j^2 - s_i^2),
//   M = F o (J - J^T) S + S F o (K - K^T) + diag(gS),
// and gB^T = Z Ut^T with Z = V_B (M^T - K S^-1) + gV_B S^-1.  This kernel writes
// M2 = M^T - K S^-1 (entries with i or j >= l, and pairs of equal singular values, zero).
__global__ void svd_adjoint_kernel(const float* __restrict__ J, const float* __restrict__ K,
                                   const float* __restrict__ s, const float* __restrict__ gS, int k,
                                   int l, int lp, float* __restrict__ M2) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= lp * lp) return;
  const int a = e / lp, b = e % lp;   // M2(a, b) = M(b, a) - K(a, b) / s_b
  float v = 0.0f;
  if (a < l && b < l) {
    const int i = b, j = a;           // M(i, j)
    if (i == j) {
      v = (gS != nullptr && i < k) ? gS[i] : 0.0f;
    } else {
      const float si = s[i], sj = s[j];
      const float d = (sj - si) * (sj + si);
      const float f = (fabsf(d) > 1e-30f) ? 1.0f / d : 0.0f;
      const float jm = J[(int64_t)i * lp + j] - J[(int64_t)j * lp + i];
      const float km = K[(int64_t)i * lp + j] - K[(int64_t)j * lp + i];
      v = f * (jm * sj + si * km);
    }
    if (b < k && s[b] > 0.0f) v -= K[(int64_t)a * lp + b] / s[b];
  }
  M2[e] = v;
}

// ---- row-wise steps --------------------------------------------------------------------

// Cotangents of the reconstruction loss ||A - U S V^T||_F^2 + sum(S) added to the caller's:
// gUt[r][j] = gU[r][j] + rec (2 s_j^2 U[r][j] - 2 s_j P[r][j]) for j < k (P = A V_B),
// zero for k <= j < lp (gU may be null).
__global__ void recon_cotangent_kernel(int64_t m, int k, int lp, const float* __restrict__ gU,
                                       const float* __restrict__ U, const float* __restrict__ P,
                                       const float* __restrict__ s, int rec, float* __restrict__ gUt) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * lp) return;
  const int64_t r = e / lp;
  const int j = (int)(e % lp);
  float v = 0.0f;
  if (j < k) {
    v = gU ? gU[r * k + j] : 0.0f;
    if (rec) v += 2.0f * s[j] * (s[j] * U[r * lp + j] - P[r * lp + j]);
  }
  gUt[e] = v;
}

// Y[r][j] = alpha X[r][j] scale_j (+ Y[r][j] when accumulate): scale_j = c_j for j < ncols
// from `c` (or 1 / c_j with inv; 1 without c), zero beyond; X leading dimension lds, Y lp.
__global__ void colscale_kernel(int64_t rows, int ncols, int lp, const float* __restrict__ X,
                                int lds, const float* __restrict__ c, int inv, float alpha,
                                int accumulate, float* __restrict__ Y) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * lp) return;
  const int64_t r = e / lp;
  const int j = (int)(e % lp);
  float v = 0.0f;
  if (j < ncols && X) {
    float sc = c ? c[j] : 1.0f;
    if (inv) sc = (sc > 0.0f) ? 1.0f / sc : 0.0f;
    v = alpha * X[r * lds + j] * sc;
  }
  Y[e] = accumulate ? Y[e] + v : v;
}

// gS_t[j] = gS[j] (or 0) + rec for j < k
__global__ void gs_total_kernel(const float* __restrict__ gS, int k, int rec, float* __restrict__ out) {
  const int j = threadIdx.x;
  if (j < k) out[j] = (gS ? gS[j] : 0.0f) + (rec ? 1.0f : 0.0f);
}

}  // namespace

cudaError_t launch_lowrank_update(int64_t m, int64_t n, int kr, const float* L, int64_t ldl,
                                  const float* R, int64_t ldr, const void* A, int64_t lda, int adt,
                                  float alpha, float beta, float* G, int64_t ldg, cudaStream_t st) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  const dim3 grid((unsigned)cdiv(n, LT), (unsigned)cdiv(m, LT));
  if (adt == 0)
    lowrank_update_kernel<0><<<grid, 256, 0, st>>>(m, n, kr, L, ldl, R, ldr, A, lda, alpha, beta, G, ldg);
  else if (adt == 1)
    lowrank_update_kernel<1><<<grid, 256, 0, st>>>(m, n, kr, L, ldl, R, ldr, A, lda, alpha, beta, G, ldg);
  else
    lowrank_update_kernel<2><<<grid, 256, 0, st>>>(m, n, kr, L, ldl, R, ldr, A, lda, alpha, beta, G, ldg);
  return cudaGetLastError();
}

cudaError_t launch_copyltu_neg(const float* C, int lp, float* N, cudaStream_t st) {
  copyltu_neg_kernel<<<(unsigned)cdiv((int64_t)lp * lp, 256), 256, 0, st>>>(C, lp, N);
  return cudaGetLastError();
}

cudaError_t launch_svd_adjoint(const float* J, const float* K, const float* s, const float* gS, int k,
                               int l, int lp, float* M2, cudaStream_t st) {
  svd_adjoint_kernel<<<(unsigned)cdiv((int64_t)lp * lp, 256), 256, 0, st>>>(J, K, s, gS, k, l, lp, M2);
  return cudaGetLastError();
}

cudaError_t launch_recon_cotangent(int64_t m, int k, int lp, const float* gU, const float* U,
                                   const float* P, const float* s, int rec, float* gUt, cudaStream_t st) {
  const int64_t n = m * lp;
  recon_cotangent_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(m, k, lp, gU, U, P, s, rec, gUt);
  return cudaGetLastError();
}

cudaError_t launch_colscale(int64_t rows, int ncols, int lp, const float* X, int lds, const float* c,
                            int inv, float alpha, int accumulate, float* Y, cudaStream_t st) {
  const int64_t n = rows * lp;
  colscale_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(rows, ncols, lp, X, lds, c, inv, alpha,
                                                           accumulate, Y);
  return cudaGetLastError();
}

cudaError_t launch_gs_total(const float* gS, int k, int rec, float* out, cudaStream_t st) {
  gs_total_kernel<<<1, 256, 0, st>>>(gS, k, rec, out);
  return cudaGetLastError();
}

}  // namespace rsvd
