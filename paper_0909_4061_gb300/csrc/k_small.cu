// Small dense products on l x l matrices (l <= 256) for the single-pass Stage B
// (Section 5.5): C = alpha op(A) op(B) + beta C, op = identity or transpose, one
// CTA per 32 x 32 block of C, K in chunks of 32 through shared memory; and the
// elementwise step of the Sylvester solve, H = G ./ (s2_i^2 + s1_j^2) (or G ./ (s2_i + s1_j)
// when the eigenvalues of the normal-equation matrices are given directly).
#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {
namespace {

constexpr int ST = 32;

__global__ void __launch_bounds__(256) small_gemm_kernel(int M, int N, int K, float alpha,
                                                         const float* __restrict__ A, int lda, int ta,
                                                         const float* __restrict__ B, int ldb, int tb,
                                                         float beta, float* __restrict__ C, int ldc) {
  __shared__ float As[ST][ST + 1];   // As[i][k] = op(A)(i0 + i, k0 + k)
  __shared__ float Bs[ST][ST + 1];   // Bs[k][j] = op(B)(k0 + k, j0 + j)
  const int i0 = blockIdx.y * ST, j0 = blockIdx.x * ST;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < K; k0 += ST) {
    for (int r = ty; r < ST; r += 8) {
      const int i = i0 + r, k = k0 + tx;
      float a = 0.0f;
      if (i < M && k < K) a = ta ? A[(int64_t)k * lda + i] : A[(int64_t)i * lda + k];
      As[r][tx] = a;
      const int kk = k0 + r, j = j0 + tx;
      float b = 0.0f;
      if (kk < K && j < N) b = tb ? B[(int64_t)j * ldb + kk] : B[(int64_t)kk * ldb + j];
      Bs[r][tx] = b;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < ST; ++k) {
      const float b = Bs[k][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(As[ty + 8 * q][k], b, acc[q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + ty + 8 * q, j = j0 + tx;
    if (i < M && j < N) {
      float* c = C + (int64_t)i * ldc + j;
      *c = alpha * acc[q] + (beta != 0.0f ? beta * *c : 0.0f);
    }
  }
}

__global__ void sylvester_scale_kernel(const float* __restrict__ G, int l, int lp,
                                       const float* __restrict__ s2, const float* __restrict__ s1,
                                       int squared, float* __restrict__ H) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= lp * lp) return;
  const int i = e / lp, j = e % lp;
  float h = 0.0f;
  if (i < l && j < l) {
    const float d = squared ? s2[i] + s1[j] : fmaf(s2[i], s2[i], s1[j] * s1[j]);
    h = d > 0.0f ? G[e] / d : 0.0f;
  }
  H[e] = h;
}

// x <- float(bf16(x)) on a rows x cols block (ld): the float32 copy of a test matrix then
// holds exactly the values the bfloat16 passes multiply with.
__global__ void round_bf16_kernel(float* __restrict__ x, int64_t rows, int cols, int64_t ld) {
  const int64_t n = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols;
    const int c = (int)(e - r * cols);
    float* p = x + r * ld + c;
    *p = __bfloat162float(__float2bfloat16_rn(*p));
  }
}

// A bounded wait on a device word that nothing sets, in the form of the library's flag
// waits (poll, back off, give up after `spins` polls and record the timeout in the status
// word): the kernel always returns, so the context stays usable.
__global__ void wait_selftest_kernel(const uint32_t* __restrict__ flag, uint32_t spins,
                                     uint32_t* __restrict__ status) {
  if (threadIdx.x != 0) return;
  const volatile uint32_t* f = flag;
  for (uint32_t i = 0; i < spins; ++i) {
    if (*f != 0u) return;
    __nanosleep(64);
  }
  set_status(status, ST_TIMEOUT);
}

// B <- (B + B^T) / 2 on the leading l x l of an lp x lp block (one thread per pair).
__global__ void symmetrize_kernel(float* __restrict__ B, int l, int lp) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= l * l) return;
  const int i = e / l, j = e % l;
  if (j <= i) return;
  const float v = 0.5f * (B[i * lp + j] + B[j * lp + i]);
  B[i * lp + j] = v;
  B[j * lp + i] = v;
}

// Eigenvalues from the SVD of a symmetric l x l matrix, X = Ut S W^T (one warp per value):
// mode 0, lambda_i = s_i sign(u_i . w_i) (the left and right singular vectors of a
// symmetric matrix agree up to the sign of its eigenvalue); mode 1, lambda_i = s_i^2.
__global__ void eig_values_kernel(const float* __restrict__ ut, const float* __restrict__ w,
                                  const float* __restrict__ s, int l, int lp, int k, int mode,
                                  float* __restrict__ out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < k; i += blockDim.x >> 5) {
    float d = 0.0f;
    if (mode == 0)
      for (int r = lane; r < l; r += 32) d = fmaf(ut[r * lp + i], w[r * lp + i], d);
    d = warp_sum(d);
    if (lane == 0) out[i] = mode == 0 ? (d < 0.0f ? -s[i] : s[i]) : s[i] * s[i];
  }
}

}  // namespace

cudaError_t launch_symmetrize(float* B, int l, int lp, cudaStream_t st) {
  symmetrize_kernel<<<(unsigned)cdiv((int64_t)l * l, 256), 256, 0, st>>>(B, l, lp);
  return cudaGetLastError();
}

cudaError_t launch_eig_values(const float* ut, const float* w, const float* s, int l, int lp, int k,
                              int mode, float* out, cudaStream_t st) {
  eig_values_kernel<<<1, 256, 0, st>>>(ut, w, s, l, lp, k, mode, out);
  return cudaGetLastError();
}

cudaError_t launch_wait_selftest(const uint32_t* flag, uint32_t spins, uint32_t* status,
                                 cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(flag, spins, status);
  return cudaGetLastError();
}

cudaError_t launch_round_bf16(float* x, int64_t rows, int cols, int64_t ld, cudaStream_t st) {
  const int64_t n = rows * cols;
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = cdiv(n, 256);
  round_bf16_kernel<<<(unsigned)(blocks < 16 * kNumSMs ? blocks : 16 * kNumSMs), 256, 0, st>>>(x, rows, cols, ld);
  return cudaGetLastError();
}

cudaError_t launch_small_gemm(int M, int N, int K, float alpha, const float* A, int lda, int ta,
                              const float* B, int ldb, int tb, float beta, float* C, int ldc,
                              cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const dim3 grid((unsigned)cdiv(N, ST), (unsigned)cdiv(M, ST));
  small_gemm_kernel<<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc);
  return cudaGetLastError();
}

cudaError_t launch_sylvester_scale(const float* G, int l, int lp, const float* s2, const float* s1,
                                   int squared, float* H, cudaStream_t st) {
  sylvester_scale_kernel<<<(unsigned)cdiv((int64_t)lp * lp, 256), 256, 0, st>>>(G, l, lp, s2, s1,
                                                                                  squared, H);
  return cudaGetLastError();
}

}  // namespace rsvd
