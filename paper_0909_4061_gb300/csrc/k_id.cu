// The interpolative decomposition of the rows of an m x l matrix Y (Section 3.2.3), with
// the rows chosen by successive orthogonalization with pivoting (Businger--Golub, Section
// 3.3.2, applied to the rows), and the gathers of Algorithm 5.2.
//
// id_pivot_kernel: one cooperative launch, one CTA per SM, each CTA owning a contiguous
// slice of rows of the residual R (initially Y).  The slice lives in shared memory while it
// fits (192 KB: m up to about 66 000 rows at l_p = 112 over 152 CTAs), a thread per row;
// beyond that it is updated in place in global memory, a warp per row.  Step i:
//   1. every CTA publishes its longest residual row (squared norm, index, the row) in a
//      double-buffered candidate slot and arrives at a grid barrier (a monotonic counter,
//      bounded spin);
//   2. every CTA picks the same winner (largest squared norm, the lowest index among
//      equal ones), v = r_w / ||r_w||, and CTA 0 records the pivot;
//   3. every row r of the slice gets c_ri = r . v (written to C[r, i]) and r <- r - c_ri v;
//      the winner's own residual is set to zero, which keeps it out of later steps.
// After l steps Y = C V^T with V = [v_1 .. v_l] orthogonal, and the chosen rows give
// Y[J] = L V^T with L = C[J] lower triangular (diagonal: the pivots' residual norms), so
// X = Y Y[J]^-1 = C L^-1: one triangular inverse of l x l and one product.
#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {
namespace {

constexpr int kIdThreads = 512;
constexpr int kIdWarps = kIdThreads / 32;
constexpr uint32_t kIdSpinLimit = 1u << 22;   // grid-barrier polls (about 0.4 s with the sleeps)
constexpr size_t kIdSliceMax = 192 * 1024;      // largest slice of rows kept in shared memory

__device__ __forceinline__ bool id_better(float n1, int r1, float n2, int r2) {
  return n1 > n2 || (n1 == n2 && r1 >= 0 && (r2 < 0 || r1 < r2));
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const unsigned* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// cand: 2 x grid slots of (4 + lp) floats: [squared norm, row index (int bits), 0, 0, row].
// SM: the CTA's slice of the residual lives in shared memory for the whole kernel (loaded
// from res at the start; res is then left as it was), else in res itself.
template <bool SM>
__global__ void __launch_bounds__(kIdThreads, 1) id_pivot_kernel(
    float* __restrict__ res, int64_t m, int l, int lp, float* __restrict__ coef,
    int* __restrict__ piv, float* __restrict__ cand, unsigned* __restrict__ bar,
    uint32_t* __restrict__ status) {
  __shared__ __align__(16) float v[kMaxL];
  __shared__ float wn[kIdWarps];
  __shared__ int wr[kIdWarps];
  __shared__ float s_best_n, s_win_n;
  __shared__ int s_best_r, s_win_r, s_win_slot, s_abort;
  const int G = gridDim.x, b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t chunk = cdiv(m, G);
  const int64_t r0 = min(m, (int64_t)b * chunk), r1 = min(m, r0 + chunk);
  const int nper = (lp + 31) / 32;   // elements of a row per lane (lp <= 256: at most 8)
  const int64_t slot_sz = 4 + lp;
  extern __shared__ __align__(16) float rows_sm[];
  // row r of the slice (r0 <= r < r1); in shared memory rows are padded to lp + 1 floats so
  // that a thread per row reads them without bank conflicts
  const int lds = lp + 1;
  auto rowp = [&](int64_t r) -> float* { return SM ? rows_sm + (r - r0) * lds : res + r * lp; };
  if (SM) {
    for (int64_t e = tid; e < (r1 - r0) * lp; e += kIdThreads) rows_sm[(e / lp) * lds + e % lp] = res[r0 * lp + e];
    __syncthreads();
  }

  // squared norms of the slice and its longest row
  float bn = -1.0f;
  int br = -1;
  for (int64_t r = r0 + warp; r < r1; r += kIdWarps) {
    const float* row = rowp(r);
    float s = 0.0f;
    for (int e = 0; e < nper; ++e) {
      const int c = lane + 32 * e;
      if (c < lp) s = fmaf(row[c], row[c], s);
    }
    s = warp_sum(s);
    if (s > 0.0f && id_better(s, (int)r, bn, br)) { bn = s; br = (int)r; }
  }
  if (lane == 0) { wn[warp] = bn; wr[warp] = br; }
  __syncthreads();
  if (tid == 0) {
    float n = -1.0f;
    int r = -1;
    for (int w = 0; w < kIdWarps; ++w)
      if (wr[w] >= 0 && id_better(wn[w], wr[w], n, r)) { n = wn[w]; r = wr[w]; }
    s_best_n = n;
    s_best_r = r;
    s_abort = 0;
  }
  __syncthreads();

  for (int i = 0; i < l; ++i) {
    // 1. publish this slice's candidate
    float* slot = cand + ((int64_t)(i & 1) * G + b) * slot_sz;
    const int myr = s_best_r;
    for (int c = tid; c < lp; c += kIdThreads) slot[4 + c] = myr >= 0 ? rowp(myr)[c] : 0.0f;
    if (tid == 0) {
      slot[0] = s_best_n;
      slot[1] = __int_as_float(myr);
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicAdd(bar, 1u);
      const uint32_t target = (uint32_t)(i + 1) * (uint32_t)G;
      uint32_t spins = 0;
      while (ld_acquire_u32(bar) < target) {
        if (++spins > kIdSpinLimit) {
          s_abort = 1;
          set_status(status, ST_TIMEOUT);
          break;
        }
        if (spins > 16) __nanosleep(64);
      }
    }
    __syncthreads();
    if (s_abort) return;
    // 2. the winner, the same in every CTA
    const float* slots = cand + (int64_t)(i & 1) * G * slot_sz;
    if (warp == 0) {
      // every lane's headers (grid <= 256: at most 8) loaded together, then compared
      float hn[8];
      int hr[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int c = lane + 32 * q;
        const float2 h = c < G ? __ldcg(reinterpret_cast<const float2*>(slots + (int64_t)c * slot_sz))
                               : make_float2(-1.0f, __int_as_float(-1));
        hn[q] = h.x;
        hr[q] = __float_as_int(h.y);
      }
      float n = -1.0f;
      int r = -1, sl = -1;
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (hr[q] >= 0 && id_better(hn[q], hr[q], n, r)) { n = hn[q]; r = hr[q]; sl = lane + 32 * q; }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float on = __shfl_xor_sync(0xffffffffu, n, o);
        const int orr = __shfl_xor_sync(0xffffffffu, r, o);
        const int osl = __shfl_xor_sync(0xffffffffu, sl, o);
        if (orr >= 0 && id_better(on, orr, n, r)) { n = on; r = orr; sl = osl; }
      }
      if (lane == 0) {
        s_win_n = n;
        s_win_r = r;
        s_win_slot = sl;
      }
    }
    __syncthreads();
    const int wrow = s_win_r;
    const float wn2 = s_win_n;
    if (wrow < 0 || !(wn2 > 0.0f) || !isfinite(wn2)) {   // Y has rank < l: no row left
      if (b == 0 && tid == 0) {
        set_status(status, ST_NUMERICAL);
        for (int t = i; t < l; ++t) piv[t] = -1;
      }
      return;
    }
    const float inv = 1.0f / sqrtf(wn2);
    const float* wvec = slots + (int64_t)s_win_slot * slot_sz + 4;
    for (int c = tid; c < lp; c += kIdThreads) v[c] = __ldcg(wvec + c) * inv;
    if (b == 0 && tid == 0) piv[i] = wrow;
    __syncthreads();
    // 3. project v out of the slice, record the coefficients, find the next candidate
    bn = -1.0f;
    br = -1;
    if (SM) {   // a thread per row
      for (int64_t r = r0 + tid; r < r1; r += kIdThreads) {
        float* row = rowp(r);
        float d0 = 0.0f, d1 = 0.0f, d2 = 0.0f, d3 = 0.0f;
        for (int c = 0; c < lp; c += 4) {   // lp is a multiple of 16
          d0 = fmaf(row[c], v[c], d0);
          d1 = fmaf(row[c + 1], v[c + 1], d1);
          d2 = fmaf(row[c + 2], v[c + 2], d2);
          d3 = fmaf(row[c + 3], v[c + 3], d3);
        }
        const float d = (d0 + d1) + (d2 + d3);
        coef[r * lp + i] = d;
        const bool win = (r == wrow);
        float s0 = 0.0f, s1 = 0.0f;
        for (int c = 0; c < lp; c += 2) {
          const float y0 = win ? 0.0f : fmaf(-d, v[c], row[c]);
          const float y1 = win ? 0.0f : fmaf(-d, v[c + 1], row[c + 1]);
          row[c] = y0;
          row[c + 1] = y1;
          s0 = fmaf(y0, y0, s0);
          s1 = fmaf(y1, y1, s1);
        }
        const float sq = s0 + s1;
        if (sq > 0.0f && id_better(sq, (int)r, bn, br)) { bn = sq; br = (int)r; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {   // the warp's best row
        const float on = __shfl_xor_sync(0xffffffffu, bn, o);
        const int orr = __shfl_xor_sync(0xffffffffu, br, o);
        if (orr >= 0 && id_better(on, orr, bn, br)) { bn = on; br = orr; }
      }
    }
    for (int64_t r = SM ? r1 : r0 + warp; r < r1; r += kIdWarps) {
      float* row = rowp(r);
      float x[8];
      float d = 0.0f;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int c = lane + 32 * e;
        x[e] = (e < nper && c < lp) ? row[c] : 0.0f;
        if (e < nper && c < lp) d = fmaf(x[e], v[c], d);
      }
      d = warp_sum(d);
      if (lane == 0) coef[r * lp + i] = d;
      const bool win = (r == wrow);
      float s = 0.0f;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int c = lane + 32 * e;
        if (e < nper && c < lp) {
          const float y = win ? 0.0f : fmaf(-d, v[c], x[e]);
          row[c] = y;
          s = fmaf(y, y, s);
        }
      }
      s = warp_sum(s);
      if (s > 0.0f && id_better(s, (int)r, bn, br)) { bn = s; br = (int)r; }
    }
    if (lane == 0) { wn[warp] = bn; wr[warp] = br; }
    __syncthreads();
    if (tid == 0) {
      float n = -1.0f;
      int r = -1;
      for (int w = 0; w < kIdWarps; ++w)
        if (wr[w] >= 0 && id_better(wn[w], wr[w], n, r)) { n = wn[w]; r = wr[w]; }
      s_best_n = n;
      s_best_r = r;
    }
    __syncthreads();
  }
}

// Lt (lp x lp, upper) = C[J]^T on the leading l x l: Lt[i][t] = C[piv[t]][i]; zero
// elsewhere (the identity where a pivot is missing).
__global__ void id_lt_kernel(const float* __restrict__ coef, const int* __restrict__ piv, int l,
                             int lp, float* __restrict__ lt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= lp * lp) return;
  const int i = e / lp, t = e % lp;
  float val = 0.0f;
  if (i < l && t < l) {
    const int pr = piv[t];
    val = pr >= 0 ? (i <= t ? coef[(int64_t)pr * lp + i] : 0.0f) : (i == t ? 1.0f : 0.0f);
  }
  lt[e] = val;
}

__global__ void transpose_square_kernel(const float* __restrict__ src, int lp, float* __restrict__ dst) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= lp * lp) return;
  const int i = e / lp, j = e % lp;
  dst[(int64_t)j * lp + i] = src[e];
}

// out (n x lp float32) = A[J, :]^T: out[c][t] = A[piv[t]][c] for t < l, zero for t >= l.
// 32 x 32 tiles through shared memory (rows of A read along c, rows of out written along t).
template <int ADT>
__global__ void gather_rows_t_kernel(const void* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                                     const int* __restrict__ piv, int l, int lp, float* __restrict__ out) {
  __shared__ float tile[32][33];
  const int64_t c0 = (int64_t)blockIdx.x * 32;
  const int t0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    const int t = t0 + k;
    const int64_t c = c0 + tx;
    float val = 0.0f;
    if (t < l && c < n) {
      const int pr = piv[t];
      if (pr >= 0) {
        if (ADT == 0) {
          val = static_cast<const float*>(A)[(int64_t)pr * lda + c];
        } else {
          const __nv_bfloat16* a = static_cast<const __nv_bfloat16*>(A);
          val = __bfloat162float(a[(int64_t)pr * lda + c]);
          if (ADT == 2) val += __bfloat162float(a[((int64_t)pr + m) * lda + c]);
        }
      }
    }
    tile[k][tx] = val;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int64_t c = c0 + k;
    const int t = t0 + tx;
    if (c < n && t < lp) out[c * lp + t] = tile[tx][k];
  }
}

}  // namespace

cudaError_t launch_id_pivot(float* res, int64_t m, int l, int lp, float* coef, int* piv, float* cand,
                            unsigned* bar, uint32_t* status, int grid, cudaStream_t st) {
  if (grid < 1 || grid > 256 || l > kMaxL || lp > kMaxL) return cudaErrorInvalidValue;
  void* args[] = {&res, &m, &l, &lp, &coef, &piv, &cand, &bar, &status};
  // the slice in shared memory when it fits beside the kernel's own arrays
  const size_t slice = (size_t)cdiv(m, grid) * (lp + 1) * sizeof(float);
  if (slice <= kIdSliceMax) {
    cudaError_t e = cudaFuncSetAttribute(id_pivot_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kIdSliceMax);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel((void*)id_pivot_kernel<true>, dim3(grid), dim3(kIdThreads), args, slice,
                                       st);
  }
  return cudaLaunchCooperativeKernel((void*)id_pivot_kernel<false>, dim3(grid), dim3(kIdThreads), args, 0, st);
}

size_t id_cand_floats(int grid, int lp) { return (size_t)2 * grid * (4 + lp); }

cudaError_t launch_id_lt(const float* coef, const int* piv, int l, int lp, float* lt, cudaStream_t st) {
  id_lt_kernel<<<(unsigned)cdiv((int64_t)lp * lp, 256), 256, 0, st>>>(coef, piv, l, lp, lt);
  return cudaGetLastError();
}

cudaError_t launch_transpose_square(const float* src, int lp, float* dst, cudaStream_t st) {
  transpose_square_kernel<<<(unsigned)cdiv((int64_t)lp * lp, 256), 256, 0, st>>>(src, lp, dst);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows_t(int adt, const void* A, int64_t lda, int64_t m, int64_t n, const int* piv,
                                 int l, int lp, float* out, cudaStream_t st) {
  const dim3 grid((unsigned)cdiv(n, 32), (unsigned)cdiv(lp, 32)), block(32, 8);
  if (adt == 0) gather_rows_t_kernel<0><<<grid, block, 0, st>>>(A, lda, m, n, piv, l, lp, out);
  else if (adt == 1) gather_rows_t_kernel<1><<<grid, block, 0, st>>>(A, lda, m, n, piv, l, lp, out);
  else gather_rows_t_kernel<2><<<grid, block, 0, st>>>(A, lda, m, n, piv, l, lp, out);
  return cudaGetLastError();
}

}  // namespace rsvd
