// Float32 CUDA-core GEMM for the plain-FP32 passes over A (Y = A X, Z = A^T X:
// Algorithm 4.4 steps 2, 4, 5 and Algorithm 5.1 step 1) and for the small
// products of the path (Q = Y R^-1 of the orthonormaliser, U = Q Ut of
// Algorithm 5.1 step 3).
//
// Tile: 128 rows x 64 columns of C per CTA, K in slabs of 16, 256 threads with
// an 8 x 4 register tile each, double-buffered shared memory with a register
// prefetch of the next slab.  The K range can be split across gridDim.z into
// partial results that a later kernel sums in a fixed order (deterministic).
#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {
namespace {

constexpr int BM = 128, BN = 64, BK = 16, NT = 256;

template <int TRANS>
struct ATile {
  float v[8];
  // trans 0: thread t loads row r = t/2, k = (t%2)*8 .. +7 of A (M x K);
  // trans 1: thread t loads k = t/16, rows (t%16)*8 .. +7 of A^T (A stored K x M).
  __device__ __forceinline__ void load(const float* __restrict__ A, int64_t lda, int64_t M,
                                       int64_t K, int64_t m0, int64_t k0, bool vec_ok) {
    const int t = threadIdx.x;
    if (TRANS == 0) {
      const int64_t r = m0 + t / 2, k = k0 + (t % 2) * 8;
      const float* p = A + r * lda + k;
      if (vec_ok && r < M && k + 8 <= K) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(p));
        const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = (r < M && k + i < K) ? __ldg(p + i) : 0.0f;
      }
    } else {
      const int64_t k = k0 + t / 16, r = m0 + (t % 16) * 8;
      const float* p = A + k * lda + r;
      if (vec_ok && k < K && r + 8 <= M) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(p));
        const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = (k < K && r + i < M) ? __ldg(p + i) : 0.0f;
      }
    }
  }
  __device__ __forceinline__ void store(float (*As)[BM + 4]) const {
    const int t = threadIdx.x;
    if (TRANS == 0) {
      const int r = t / 2, k = (t % 2) * 8;
#pragma unroll
      for (int i = 0; i < 8; ++i) As[k + i][r] = v[i];
    } else {
      const int k = t / 16, r = (t % 16) * 8;
      *reinterpret_cast<float4*>(&As[k][r]) = make_float4(v[0], v[1], v[2], v[3]);
      *reinterpret_cast<float4*>(&As[k][r + 4]) = make_float4(v[4], v[5], v[6], v[7]);
    }
  }
};

struct XTile {
  float v[4];
  // thread t loads k = t/16, columns (t%16)*4 .. +3 of X (K x N).
  __device__ __forceinline__ void load(const float* __restrict__ X, int64_t ldx, int64_t N,
                                       int64_t K, int64_t n0, int64_t k0, bool vec_ok) {
    const int t = threadIdx.x;
    const int64_t k = k0 + t / 16, c = n0 + (t % 16) * 4;
    const float* p = X + k * ldx + c;
    if (vec_ok && k < K && c + 4 <= N) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(p));
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] = (k < K && c + i < N) ? __ldg(p + i) : 0.0f;
    }
  }
  __device__ __forceinline__ void store(float (*Xs)[BN]) const {
    const int t = threadIdx.x;
    *reinterpret_cast<float4*>(&Xs[t / 16][(t % 16) * 4]) = make_float4(v[0], v[1], v[2], v[3]);
  }
};

template <int TRANS>
__global__ void __launch_bounds__(NT) gemm_f32_kernel(int64_t M, int64_t N, int64_t K,
                                                      const float* __restrict__ A, int64_t lda,
                                                      const float* __restrict__ X, int64_t ldx,
                                                      float* __restrict__ C, int64_t ldc,
                                                      int splits, int64_t split_stride,
                                                      int a_vec, int x_vec) {
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Xs[2][BK][BN];

  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int64_t n0 = (int64_t)blockIdx.y * BN;
  const int s = blockIdx.z;
  const int64_t kt = cdiv(K, BK);
  const int64_t kb = kt * s / splits, ke = kt * (s + 1) / splits;
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;

  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;

  ATile<TRANS> at;
  XTile xt;
  if (kb < ke) {
    at.load(A, lda, M, K, m0, kb * BK, a_vec);
    xt.load(X, ldx, N, K, n0, kb * BK, x_vec);
    at.store(As[0]);
    xt.store(Xs[0]);
  }
  __syncthreads();
  int buf = 0;
  for (int64_t kk = kb; kk < ke; ++kk) {
    const bool more = kk + 1 < ke;
    if (more) {
      at.load(A, lda, M, K, m0, (kk + 1) * BK, a_vec);
      xt.load(X, ldx, N, K, n0, (kk + 1) * BK, x_vec);
    }
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 8 + 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Xs[buf][k][tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (more) {
      at.store(As[buf ^ 1]);
      xt.store(Xs[buf ^ 1]);
    }
    __syncthreads();
    buf ^= 1;
  }

  float* Cs = C + (int64_t)s * split_stride;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t r = m0 + ty * 8 + i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t c = n0 + tx * 4 + j;
      if (c < N) Cs[r * ldc + c] = acc[i][j];
    }
  }
}

}  // namespace

cudaError_t launch_gemm_f32(int trans, int64_t M, int64_t N, int64_t K, const float* A,
                            int64_t lda, const float* X, int64_t ldx, float* C, int64_t ldc,
                            int splits, int64_t split_stride, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (splits < 1) splits = 1;
  const dim3 grid((unsigned)cdiv(M, BM), (unsigned)cdiv(N, BN), (unsigned)splits);
  const int a_vec = ((reinterpret_cast<uintptr_t>(A) & 15) == 0) && (lda % 4 == 0);
  const int x_vec = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && (ldx % 4 == 0);
  if (trans)
    gemm_f32_kernel<1><<<grid, NT, 0, st>>>(M, N, K, A, lda, X, ldx, C, ldc, splits, split_stride,
                                            a_vec, x_vec);
  else
    gemm_f32_kernel<0><<<grid, NT, 0, st>>>(M, N, K, A, lda, X, ldx, C, ldc, splits, split_stride,
                                            a_vec, x_vec);
  return cudaGetLastError();
}

}  // namespace rsvd
