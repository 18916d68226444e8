// The SRFT sketch as a transform along the rows of A (Section 4.6, Algorithm 4.5 step 2):
// Y = A Omega with Omega = sqrt(n / l_c) D F R, i.e. for every row a of A
//     y_c = l_c^-1/2 sum_j a_j d_j exp(-2 pi i j b_c / n)        (c = 0 .. l_c - 1),
// stored as the real columns [Re y_c, Im y_c] (the real form of the SRFT test matrix
// used throughout the library; d_j = +-1, b_c the sampled frequencies).
//
// One CTA transforms one row at a time in shared memory.  The row is real of length
// n = 2N, so it is packed into the complex sequence z_j = x_{2j} + i x_{2j+1} (x = a d) of
// length N, whose DFT Z gives the real DFT by the usual split
//     X(b) = (Z(b) + conj Z(N - b)) / 2 - i W_n^b (Z(b) - conj Z(N - b)) / 2.
// Z comes from the four-step factorisation N = N1 N2 (j = N2 j1 + j2, k = k1 + N1 k2):
//   1. for every column j2: a length-N1 DFT over j1 (one warp),
//   2. the twiddle W_N^(j2 k1),
//   3. for every row k1: a length-N2 DFT over j2 (one warp),
// each DFT of length L = 32 R split as R x 32: a length-R DFT in every lane's registers,
// the twiddle W_L^(lane k_r), and a length-32 DFT across the lanes (five radix-2 stages by
// shuffles, outputs in bit-reversed lane order).  Only the 2 l_c entries of Z that the
// sampled frequencies need are read back.  Twiddles come from two small tables (W_N^t =
// W_N^(t mod N2) W_N1^(t div N2)), built once per CTA by sincospif.
//
// Sizes: n a power of two, 2048 <= n <= 32768 (N1, N2 in {32, 64, 128}); the row buffer is
// N1 x (N2 + 1) float2 (132 KB at n = 32768; the padding spreads a column over the banks).
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"
#include "philox.cuh"

namespace rsvd {
namespace {

constexpr int kFftThreads = 512;
constexpr int kFftWarps = kFftThreads / 32;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 shfl_xor2(float2 v, int m) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

__device__ __forceinline__ int bitrev5(int x) { return (int)(__brev((unsigned)x) >> 27); }

// Length-32 DFT across the lanes (v = element `lane`), radix-2 decimation in frequency:
// on return lane l holds X(bitrev5(l)).  w32[t] = W_32^t.
__device__ __forceinline__ float2 dft32_lanes(float2 v, int lane, const float2* __restrict__ w32) {
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const float2 u = shfl_xor2(v, h);
    if ((lane & h) == 0) {
      v = cadd(v, u);
    } else {
      v = cmul(csub(u, v), w32[(lane & (h - 1)) * (16 / h)]);   // W_{2h}^(i mod 2h)
    }
  }
  return v;
}

// Length-L DFT, L = 32 R, of the sequence whose element e = lane + 32 t is v[t]: on return
// v[kr] = X(kr + R bitrev5(lane)).  wL[t] = W_L^t (t < L), w32 as above.
template <int R>
__device__ __forceinline__ void dft_warp(float2 (&v)[R], int lane, const float2* __restrict__ wL,
                                         const float2* __restrict__ w32) {
  // length-R DFT over t in registers: y[kr] = sum_t v[t] W_R^(t kr)
  float2 y[R];
  if (R == 1) {
    y[0] = v[0];
  } else if (R == 2) {
    y[0] = cadd(v[0], v[1]);
    y[1] = csub(v[0], v[1]);
  } else {   // R == 4: W_4 = -i
    const float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    const float2 s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
    y[0] = cadd(s02, s13);
    y[2] = csub(s02, s13);
    y[1] = make_float2(d02.x + d13.y, d02.y - d13.x);   // d02 - i d13
    y[3] = make_float2(d02.x - d13.y, d02.y + d13.x);   // d02 + i d13
  }
#pragma unroll
  for (int kr = 0; kr < R; ++kr) {
    const float2 t = kr == 0 ? y[0] : cmul(y[kr], wL[lane * kr]);   // W_L^(lane kr)
    v[kr] = dft32_lanes(t, lane, w32);
  }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Rows are loaded in one of two ways.  STAGE (bfloat16 A with 16-byte aligned rows): the next
// row is copied into a shared-memory stage by cp.async while the current one is
// transformed.  Otherwise every thread loads its share of the row in batches of eight, all
// in flight at once.
template <int R1, int R2, int ADT, bool STAGE>
__global__ void __launch_bounds__(kFftThreads, 1) srft_fft_kernel(
    const void* __restrict__ A, int64_t lda, int64_t m, const uint32_t* __restrict__ signs,
    const int* __restrict__ freq, int lc, float* __restrict__ y, int ldy) {
  constexpr int N1 = 32 * R1, N2 = 32 * R2, N = N1 * N2, n = 2 * N;
  constexpr int LD = N2 + 1;   // padded row of the N1 x N2 buffer
  extern __shared__ float2 fsm[];
  float2* F = fsm;                          // N1 x LD
  float2* wN2 = F + N1 * LD;                // W_N^t, t < N2
  float2* wN1 = wN2 + N2;                   // W_N1^t, t < N1  (= W_N^(N2 t))
  float2* wL1 = wN1 + N1;                   // W_N1^t (column DFTs)
  float2* wL2 = wL1 + N1;                   // W_N2^t (row DFTs)
  float2* w32 = wL2 + N2;                   // W_32^t
  float2* wb = w32 + 32;                    // W_n^(b_c), c < lc
  uint32_t* sg = reinterpret_cast<uint32_t*>(wb + 1024);   // the n sign bits
  __nv_bfloat162* stage = reinterpret_cast<__nv_bfloat162*>(sg + n / 32);   // STAGE: one row
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int t = tid; t < n / 32; t += kFftThreads) sg[t] = signs[t];
  auto stage_row = [&](int64_t rr) {   // STAGE: the bfloat16 row rr into `stage` (N words)
    const uint4* src = reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(A) + rr * lda);
    for (int e = tid; e < N / 4; e += kFftThreads) cp_async16(stage + 4 * e, src + e);
    cp_async_commit();
  };
  if (STAGE && (int64_t)blockIdx.x < m) stage_row(blockIdx.x);
  for (int t = tid; t < N2; t += kFftThreads) {
    float s, c;
    sincospif(-2.0f * (float)t / (float)N, &s, &c);
    wN2[t] = make_float2(c, s);
    sincospif(-2.0f * (float)t / (float)N2, &s, &c);
    wL2[t] = make_float2(c, s);
  }
  for (int t = tid; t < N1; t += kFftThreads) {
    float s, c;
    sincospif(-2.0f * (float)t / (float)N1, &s, &c);
    wN1[t] = make_float2(c, s);
    wL1[t] = make_float2(c, s);
  }
  for (int t = tid; t < 32; t += kFftThreads) {
    float s, c;
    sincospif(-(float)t / 16.0f, &s, &c);
    w32[t] = make_float2(c, s);
  }
  for (int c = tid; c < lc; c += kFftThreads) {
    float s, cs;
    sincospif(-2.0f * (float)freq[c] / (float)n, &s, &cs);
    wb[c] = make_float2(cs, s);
  }
  const float scale = rsqrtf((float)lc);
  // z_j = d_2j a_2j + i d_2j+1 a_2j+1 into F[j / N2][j % N2]
  auto put = [&](int j, float a0, float a1) {
    const uint32_t w = sg[(2 * j) >> 5];
    const int sh = (2 * j) & 31;
    if ((w >> sh) & 1u) a0 = -a0;
    if ((w >> (sh + 1)) & 1u) a1 = -a1;
    F[(j / N2) * LD + (j % N2)] = make_float2(a0, a1);
  };
  for (int64_t r = blockIdx.x; r < m; r += gridDim.x) {
    if (STAGE) cp_async_wait_all();
    __syncthreads();   // the row is staged; the previous row's reads of F are done
    if (STAGE) {
      for (int j = tid; j < N; j += kFftThreads) {
        const float2 p = __bfloat1622float2(stage[j]);
        put(j, p.x, p.y);
      }
      __syncthreads();   // the stage is free: the next row streams in during this one
      if (r + gridDim.x < m) stage_row(r + gridDim.x);
    } else {
      constexpr int B = 8;
      for (int j0 = tid; j0 < N; j0 += B * kFftThreads) {
        float2 p[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
          const int j = j0 + u * kFftThreads;
          if (j >= N) break;
          if (ADT == 0) {
            p[u] = reinterpret_cast<const float2*>(static_cast<const float*>(A) + r * lda)[j];
          } else {
            const __nv_bfloat162* row = reinterpret_cast<const __nv_bfloat162*>(
                static_cast<const __nv_bfloat16*>(A) + r * lda);
            p[u] = __bfloat1622float2(row[j]);
            if (ADT == 2) {   // the residual lo, m rows further
              const __nv_bfloat162* lo = reinterpret_cast<const __nv_bfloat162*>(
                  static_cast<const __nv_bfloat16*>(A) + (m + r) * lda);
              const float2 q = __bfloat1622float2(lo[j]);
              p[u].x += q.x;
              p[u].y += q.y;
            }
          }
        }
#pragma unroll
        for (int u = 0; u < B; ++u) {
          const int j = j0 + u * kFftThreads;
          if (j < N) put(j, p[u].x, p[u].y);
        }
      }
      __syncthreads();
    }
    // The DFTs leave lane l holding output kr + R bitrev5(l) in its register kr; storing it
    // at position 32 kr + l (the transform's order, not the natural one) keeps every store
    // conflict-free.  pos(k) = 32 (k mod R) + bitrev5(k div R) maps an output index to it.
    // 1 + 2: column DFTs over j1 (length N1), the twiddle W_N^(j2 k1), into row pos(k1)
    for (int j2 = warp; j2 < N2; j2 += kFftWarps) {
      float2 v[R1];
#pragma unroll
      for (int t = 0; t < R1; ++t) v[t] = F[(lane + 32 * t) * LD + j2];
      dft_warp<R1>(v, lane, wL1, w32);
      const int br = bitrev5(lane);
#pragma unroll
      for (int kr = 0; kr < R1; ++kr) {
        const int k1 = kr + R1 * br;
        const int e = j2 * k1;   // < N: W_N^e = W_N^(e mod N2) W_N1^(e div N2)
        const float2 tw = cmul(wN2[e % N2], wN1[e / N2]);
        F[(32 * kr + lane) * LD + j2] = cmul(v[kr], tw);
      }
    }
    __syncthreads();
    // 3: row DFTs over j2 (length N2): Z(k1 + N1 k2) at row pos(k1), column pos(k2)
    for (int p1 = warp; p1 < N1; p1 += kFftWarps) {
      float2 v[R2];
#pragma unroll
      for (int t = 0; t < R2; ++t) v[t] = F[p1 * LD + lane + 32 * t];
      dft_warp<R2>(v, lane, wL2, w32);
      __syncwarp();
#pragma unroll
      for (int kr = 0; kr < R2; ++kr) F[p1 * LD + 32 * kr + lane] = v[kr];
    }
    __syncthreads();
    // the sampled frequencies: X(b) from Z(b) and Z(N - b), 1 <= b < N
    auto zat = [&](int k) {
      const int k1 = k % N1, k2 = k / N1;
      const int p1 = 32 * (k1 % R1) + bitrev5(k1 / R1), p2 = 32 * (k2 % R2) + bitrev5(k2 / R2);
      return F[p1 * LD + p2];
    };
    float* yr = y + r * (int64_t)ldy;
    for (int c = tid; c < lc; c += kFftThreads) {
      const int b = freq[c], bm = N - b;
      const float2 zb = zat(b);
      const float2 zc = cconj(zat(bm));
      const float2 e = make_float2(0.5f * (zb.x + zc.x), 0.5f * (zb.y + zc.y));
      const float2 d = make_float2(0.5f * (zb.x - zc.x), 0.5f * (zb.y - zc.y));
      const float2 o = cmul(wb[c], make_float2(d.y, -d.x));   // W_n^b (d / i)
      yr[2 * c] = scale * (e.x + o.x);
      yr[2 * c + 1] = scale * (e.y + o.y);
    }
    for (int c = 2 * lc + tid; c < ldy; c += kFftThreads) yr[c] = 0.0f;
  }
}

// d_j = -1 where bit j of the mask is set: the top bit of word j mod 4 of the Philox block
// (j / 4, 0, 2, 0) of the SRFT draws (as srft_omega_kernel reads them).
__global__ void srft_signs_kernel(uint2 key, int64_t n, uint32_t* __restrict__ mask) {
  const int64_t wi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (wi * 32 >= n) return;
  uint32_t bits = 0;
  for (int t = 0; t < 32; ++t) {
    const int64_t j = wi * 32 + t;
    if (j >= n) break;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)(j >> 2), 0u, 2u, 0u), key);
    const uint32_t q = (uint32_t)(j & 3);
    const uint32_t x = q == 0 ? w.x : (q == 1 ? w.y : (q == 2 ? w.z : w.w));
    bits |= (x >> 31) << t;
  }
  mask[wi] = bits;
}

template <int R1, int R2>
size_t fft_smem(bool stage) {
  constexpr int N1 = 32 * R1, N2 = 32 * R2, N = N1 * N2;
  return sizeof(float2) * ((size_t)N1 * (N2 + 1) + 2 * N2 + 2 * N1 + 32 + 1024) +
         sizeof(uint32_t) * (2 * N / 32) + (stage ? sizeof(uint32_t) * N : 0);
}

template <int R1, int R2, int ADT, bool STAGE>
cudaError_t launch_one(const void* A, int64_t lda, int64_t m, const uint32_t* signs, const int* freq,
                       int lc, float* y, int ldy, int grid, cudaStream_t st) {
  const size_t sm = fft_smem<R1, R2>(STAGE);
  cudaError_t e = cudaFuncSetAttribute(srft_fft_kernel<R1, R2, ADT, STAGE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  srft_fft_kernel<R1, R2, ADT, STAGE><<<grid, kFftThreads, sm, st>>>(A, lda, m, signs, freq, lc, y, ldy);
  return cudaGetLastError();
}

template <int R1, int R2>
cudaError_t launch_rr(int adt, const void* A, int64_t lda, int64_t m, const uint32_t* signs,
                      const int* freq, int lc, float* y, int ldy, int grid, cudaStream_t st) {
  // the stage takes 16-byte copies: rows must start on 16-byte boundaries
  const bool stage = adt == 1 && (reinterpret_cast<uintptr_t>(A) & 15) == 0 && (lda % 8) == 0;
  if (adt == 0) return launch_one<R1, R2, 0, false>(A, lda, m, signs, freq, lc, y, ldy, grid, st);
  if (adt == 2) return launch_one<R1, R2, 2, false>(A, lda, m, signs, freq, lc, y, ldy, grid, st);
  if (stage) return launch_one<R1, R2, 1, true>(A, lda, m, signs, freq, lc, y, ldy, grid, st);
  return launch_one<R1, R2, 1, false>(A, lda, m, signs, freq, lc, y, ldy, grid, st);
}

}  // namespace

bool srft_fft_supported(int64_t n) {
  return n >= 2048 && n <= 32768 && (n & (n - 1)) == 0;
}

cudaError_t launch_srft_signs(uint64_t seed, int64_t n, uint32_t* mask, cudaStream_t st) {
  const int64_t words = cdiv(n, 32);
  srft_signs_kernel<<<(unsigned)cdiv(words, 256), 256, 0, st>>>(seed_key(seed), n, mask);
  return cudaGetLastError();
}

cudaError_t launch_srft_fft(int adt, const void* A, int64_t lda, int64_t m, int64_t n,
                            const uint32_t* signs, const int* freq, int lc, float* y, int ldy,
                            int num_sms, cudaStream_t st) {
  if (!srft_fft_supported(n) || lc < 1 || lc > 1024 || 2 * lc > ldy || m < 1) return cudaErrorInvalidValue;
  // the bfloat16 pairs and float2 loads need an even leading dimension
  if (lda % 2) return cudaErrorInvalidValue;
  const int grid = (int)(m < num_sms ? m : num_sms);
  const int64_t N = n / 2;   // N1 x N2, N1 <= N2, both in {32, 64, 128}
  switch (N) {
    case 1024: return launch_rr<1, 1>(adt, A, lda, m, signs, freq, lc, y, ldy, grid, st);
    case 2048: return launch_rr<1, 2>(adt, A, lda, m, signs, freq, lc, y, ldy, grid, st);
    case 4096: return launch_rr<2, 2>(adt, A, lda, m, signs, freq, lc, y, ldy, grid, st);
    case 8192: return launch_rr<2, 4>(adt, A, lda, m, signs, freq, lc, y, ldy, grid, st);
    default: return launch_rr<4, 4>(adt, A, lda, m, signs, freq, lc, y, ldy, grid, st);
  }
}

}  // namespace rsvd
