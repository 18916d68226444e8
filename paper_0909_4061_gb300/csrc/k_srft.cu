// Subsampled random Fourier transform test matrix (Section 4.6, Algorithm 4.5
// step 1), Omega = sqrt(n / l_c) D F R, for a real A.
//
// D: random signs d_i = +-1; F: the unitary n-point DFT, f_pq = n^-1/2
// exp(-2 pi i p q / n) (0-based); R: l_c frequencies drawn without replacement.
// A is real, so the columns of A D F at b and n - b are complex conjugates: the
// frequencies come from {1, ..., n/2 - 1} (one per conjugate pair; 0 and n/2 are
// self-conjugate) and the real test matrix interleaves [Re w_c, Im w_c], n x 2 l_c,
// which spans the same real space as the complex samples at b_c and n - b_c.
//
// The sketch Y = A Omega is then an ordinary pass over A on the tensor cores.
// Applying F by an FFT would save arithmetic, not memory traffic, and a pass over A
// is bound by HBM here at l <= 256 (l flop per byte of bf16 A, against a ridge near
// 300), so the structured matrix is materialised (n x l, a few MB) instead.
//
// Draws (Philox4x32-10, stream 2): d_i is the top bit of word i mod 4 of counter
// (i / 4, 0, 2, 0); candidate b has key word b mod 4 of counter (b / 4, 1, 2, 0);
// the l_c candidates with the smallest (key, b) are taken in ascending order.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"
#include "philox.cuh"

namespace rsvd {
namespace {

constexpr uint32_t kStreamSrft = 2u;
constexpr int kSelThreads = 1024;
constexpr int kSelN = 2048;   // merge buffer: best (<= 1024 kept) + one chunk of 1024

__device__ __forceinline__ uint32_t srft_word(uint2 key, uint32_t row, uint64_t idx) {
  const uint4 w = philox4x32_10(make_uint4((uint32_t)(idx >> 2), row, kStreamSrft, 0u), key);
  const uint32_t q = (uint32_t)(idx & 3u);
  return q == 0 ? w.x : (q == 1 ? w.y : (q == 2 ? w.z : w.w));
}

// One CTA: keep the lc smallest (key << 32 | b) seen so far; each chunk of 1024
// candidates is sorted together with them (bitonic network on 2048 entries).
__global__ void __launch_bounds__(kSelThreads) srft_select_kernel(uint2 key, int64_t n, int lc,
                                                                  int* __restrict__ freq) {
  __shared__ unsigned long long buf[kSelN];
  const int tid = threadIdx.x;
  const int64_t ncand = n / 2 - 1;   // b = 1 .. n/2 - 1
  for (int e = tid; e < kSelN; e += kSelThreads) buf[e] = ~0ull;
  __syncthreads();
  for (int64_t c0 = 0; c0 < ncand; c0 += kSelThreads) {
    const int64_t b = 1 + c0 + tid;
    unsigned long long v = ~0ull;
    if (b <= ncand) v = ((unsigned long long)srft_word(key, 1u, (uint64_t)b) << 32) | (unsigned long long)b;
    // the kept entries sit in buf[0 .. lc), sorted; the chunk goes to the upper half
    buf[kSelThreads + tid] = v;
    for (int e = lc + tid; e < kSelThreads; e += kSelThreads) buf[e] = ~0ull;
    __syncthreads();
    for (int size = 2; size <= kSelN; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int e = tid; e < kSelN / 2; e += kSelThreads) {
          const int lo = 2 * e - (e & (stride - 1));
          const int hi = lo + stride;
          const bool up = ((lo & size) == 0);
          const unsigned long long x = buf[lo], y = buf[hi];
          if ((x > y) == up) { buf[lo] = y; buf[hi] = x; }
        }
        __syncthreads();
      }
    }
  }
  for (int e = tid; e < lc; e += kSelThreads) freq[e] = (int)(buf[e] & 0xffffffffu);
}

// Omega (n x cols_pad, ld) and optionally its transposed bf16 copy: column 2c / 2c + 1
// = d_i cos / sin(-2 pi (i b_c mod n) / n) / sqrt(l_c); columns >= 2 l_c are zero.
__global__ void srft_omega_kernel(uint2 key, int64_t n, int lc, int cols_pad,
                                  const int* __restrict__ freq, float* __restrict__ out, int64_t ld,
                                  __nv_bfloat16* __restrict__ out_t, int64_t ld_t) {
  const float scale = rsqrtf((float)lc);
  const int64_t total = n * cols_pad;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n;   // consecutive threads take consecutive rows
    const int j = (int)(e / n);
    float val = 0.0f;
    if (j < 2 * lc) {
      const int64_t b = freq[j >> 1];
      int64_t r = (int64_t)(((unsigned long long)i * (unsigned long long)b) % (unsigned long long)n);
      if (2 * r > n) r -= n;   // same angle, reduced to [-pi, pi]
      const float x = -2.0f * (float)r / (float)n;
      float sv, cv;
      sincospif(x, &sv, &cv);
      const float d = (srft_word(key, 0u, (uint64_t)i) >> 31) ? -scale : scale;
      val = d * ((j & 1) ? sv : cv);
    }
    if (out) out[i * ld + j] = val;
    if (out_t) out_t[(int64_t)j * ld_t + i] = __float2bfloat16_rn(val);
  }
}

// ---- the modified SRFT (Section 4.6, eq. random_Givens): Omega_G = D'' Theta' D' Theta
// Omega with Omega the SRFT above and Theta = Pi G(1, 2; t_1) ... G(n-1, n; t_{n-1}),
// G(i, i+1; t) = [[c, s], [-s, c]] in rows/columns (i, i+1), (Pi x)_k = x_perm[k].
// Draws on stream 2: rows 2, 3 signs d', d''; rows 4, 6 the keys of Pi, Pi' (perm lists
// the indices by ascending (key, index)); rows 5, 7 the angles, t_i = 2 pi u_i with
// u_i = (word >> 8) 2^-24.

// rank of (key_j, j) among all n pairs = the position of j in the permutation.  Each
// thread ranks one index against the keys, staged 2048 at a time in shared memory.
constexpr int kRankTile = 2048;

__global__ void __launch_bounds__(256) gsrft_perm_kernel(uint2 key, int64_t n, uint32_t row,
                                                         int* __restrict__ perm) {
  __shared__ uint32_t ks[kRankTile];
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t kj = j < n ? srft_word(key, row, (uint64_t)j) : 0u;
  int64_t rank = 0;
  for (int64_t t0 = 0; t0 < n; t0 += kRankTile) {
    __syncthreads();
    for (int e = threadIdx.x; e < kRankTile; e += blockDim.x)
      if (t0 + e < n) ks[e] = srft_word(key, row, (uint64_t)(t0 + e));
    __syncthreads();
    const int cnt = (int)min((int64_t)kRankTile, n - t0);
    if (j < n) {
      for (int e = 0; e < cnt; ++e) {
        const uint32_t k = ks[e];
        rank += (k < kj) || (k == kj && t0 + e < j);
      }
    }
  }
  if (j < n) perm[rank] = (int)j;
}

// cos / sin of the rotation angles of both chains, once per plan: cs[chain][i] for the
// rotation in plane (i, i + 1), i < n - 1 (float32 sincospi of the exactly representable
// 2 u_i).
__global__ void gsrft_angles_kernel(uint2 key, int64_t n, float2* __restrict__ cs) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 2 * (n - 1);
       e += (int64_t)gridDim.x * blockDim.x) {
    const int chain = (int)(e / (n - 1));
    const int64_t i = e % (n - 1);
    const float u = (float)(srft_word(key, chain ? 7u : 5u, (uint64_t)i) >> 8) * 5.9604644775390625e-08f;
    float sn, cn;
    sincospif(2.0f * u, &sn, &cn);
    cs[chain * n + i] = make_float2(cn, sn);
  }
}

// dst = G(1, 2; t_1) ... G(n-1, n; t_{n-1}) src on the columns c < ncols (n x ld), the
// rightmost rotation first.  Rotation i maps the running value r of row i + 1 and v_i to
//   dst_{i+1} = -s_i v_i + c_i r,   r <- c_i v_i + s_i r,
// a first-order linear recurrence, so the chain is split into 32 segments of rotations,
// one warp each (lane = column: coalesced rows).  Pass 1: every segment's map of its
// incoming running value, r_out = alpha r_in + beta.  Then warp 0 carries the true value
// from the top (r = src_{n-1}) down the segments, and pass 2 recomputes each segment with
// its incoming value and writes its rows.
constexpr int kChainSeg = 32;

__global__ void __launch_bounds__(32 * kChainSeg) gsrft_chain_kernel(
    int64_t n, const float2* __restrict__ cs, const float* __restrict__ src, float* __restrict__ dst,
    int64_t ld, int ncols) {
  __shared__ float s_alpha[kChainSeg][32], s_beta[kChainSeg][32], s_in[kChainSeg][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + lane;
  const bool live = c < ncols;
  const int64_t nrot = n - 1, seg = cdiv(nrot, kChainSeg);
  const int64_t a = min(nrot, (int64_t)w * seg), b = min(nrot, a + seg);
  float alpha = 1.0f, beta = 0.0f;
#pragma unroll 4
  for (int64_t i = b - 1; i >= a; --i) {
    const float2 t = cs[i];
    const float v = live ? src[i * ld + c] : 0.0f;
    alpha *= t.y;
    beta = fmaf(t.x, v, t.y * beta);
  }
  s_alpha[w][lane] = alpha;
  s_beta[w][lane] = beta;
  __syncthreads();
  if (w == 0) {
    float r = live ? src[(n - 1) * ld + c] : 0.0f;
    for (int j = kChainSeg - 1; j >= 0; --j) {
      s_in[j][lane] = r;
      r = fmaf(s_alpha[j][lane], r, s_beta[j][lane]);
    }
  }
  __syncthreads();
  float r = s_in[w][lane];
#pragma unroll 4
  for (int64_t i = b - 1; i >= a; --i) {
    const float2 t = cs[i];
    const float v = live ? src[i * ld + c] : 0.0f;
    if (live) dst[(i + 1) * ld + c] = fmaf(-t.y, v, t.x * r);
    r = fmaf(t.x, v, t.y * r);
  }
  if (w == 0 && live) dst[c] = r;
}

// dst[k][c] = d_k src[perm[k]][c] for c < ncols (d from the sign row), zero for
// ncols <= c < cols_pad.
__global__ void gsrft_permute_kernel(uint2 key, int64_t n, uint32_t sign_row, const int* __restrict__ perm,
                                     const float* __restrict__ src, float* __restrict__ dst, int64_t ld,
                                     int ncols, int cols_pad) {
  const int64_t total = n * cols_pad;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e / cols_pad;
    const int c = (int)(e % cols_pad);
    float v = 0.0f;
    if (c < ncols) {
      v = src[(int64_t)perm[k] * ld + c];
      if (srft_word(key, sign_row, (uint64_t)k) >> 31) v = -v;
    }
    dst[k * ld + c] = v;
  }
}

}  // namespace

cudaError_t launch_gsrft_prepare(uint64_t seed, int64_t n, int* tables, cudaStream_t st) {
  if (n < 2 || n >= (int64_t)1 << 24) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)cdiv(n, 256);
  gsrft_perm_kernel<<<grid, 256, 0, st>>>(seed_key(seed), n, 4u, tables);
  gsrft_perm_kernel<<<grid, 256, 0, st>>>(seed_key(seed), n, 6u, tables + n);
  gsrft_angles_kernel<<<(unsigned)std::min<int64_t>(cdiv(2 * n, 256), 16 * kNumSMs), 256, 0, st>>>(
      seed_key(seed), n, reinterpret_cast<float2*>(tables + 2 * n));
  return cudaGetLastError();
}

size_t gsrft_table_ints(int64_t n) { return (size_t)6 * n; }

cudaError_t launch_gsrft_apply(uint64_t seed, int64_t n, int ncols, int cols_pad, const int* tables,
                               float* omega, float* scratch, int64_t ld, cudaStream_t st) {
  if (n < 2 || ncols < 1 || ncols > cols_pad || cols_pad > ld) return cudaErrorInvalidValue;
  const uint2 key = seed_key(seed);
  const unsigned gc = (unsigned)cdiv(ncols, 32);
  const int64_t total = n * cols_pad;
  const unsigned gp = (unsigned)std::min<int64_t>(cdiv(total, 256), 16 * kNumSMs);
  const float2* cs = reinterpret_cast<const float2*>(tables + 2 * n);
  gsrft_chain_kernel<<<gc, 32 * kChainSeg, 0, st>>>(n, cs, omega, scratch, ld, ncols);       // G chain
  gsrft_permute_kernel<<<gp, 256, 0, st>>>(key, n, 2u, tables, scratch, omega, ld, ncols, cols_pad);  // D' Pi
  gsrft_chain_kernel<<<gc, 32 * kChainSeg, 0, st>>>(n, cs + n, omega, scratch, ld, ncols);  // G' chain
  gsrft_permute_kernel<<<gp, 256, 0, st>>>(key, n, 3u, tables + n, scratch, omega, ld, ncols, cols_pad);  // D'' Pi'
  return cudaGetLastError();
}

cudaError_t launch_srft_select(uint64_t seed, int64_t n, int lc, int* freq, cudaStream_t st) {
  if (n < 4 || (n & 1) || lc < 1 || lc > n / 2 - 1 || lc > kSelThreads) return cudaErrorInvalidValue;
  srft_select_kernel<<<1, kSelThreads, 0, st>>>(seed_key(seed), n, lc, freq);
  return cudaGetLastError();
}

cudaError_t launch_draw_srft(uint64_t seed, int64_t n, int lc, int cols_pad, const int* freq,
                             float* out, int64_t ld, __nv_bfloat16* out_t, int64_t ld_t,
                             cudaStream_t st) {
  if (n <= 0 || cols_pad < 2 * lc || n >= (int64_t)1 << 24) return cudaErrorInvalidValue;
  const int64_t total = n * cols_pad;
  const int64_t blocks = cdiv(total, 256);
  const unsigned grid = (unsigned)(blocks < 16 * kNumSMs ? blocks : 16 * kNumSMs);
  srft_omega_kernel<<<grid, 256, 0, st>>>(seed_key(seed), n, lc, cols_pad, freq, out, ld, out_t, ld_t);
  return cudaGetLastError();
}

}  // namespace rsvd
