// The interpolative decomposition of the rows of an m x l matrix Y (Section 3.2.3), with
// the rows chosen by successive orthogonalization with pivoting (Businger--Golub, Section
// 3.3.2, applied to the rows), and the gathers of Algorithm 5.2.
//
// id_pivot_kernel: one cooperative launch, one CTA per SM, each CTA owning a contiguous
// slice of rows of the residual R (initially Y, updated in place in global memory: it is
// read and written once per step, from L2 at the sizes of the path).  Step i:
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

__device__ __forceinline__ bool id_better(float n1, int r1, float n2, int r2) {
  return n1 > n2 || (n1 == n2 && r1 >= 0 && (r2 < 0 || r1 < r2));
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const unsigned* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// cand: 2 x grid slots of (4 + lp) floats: [squared norm, row index (int bits), 0, 0, row].
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

  // squared norms of the slice and its longest row
  float bn = -1.0f;
  int br = -1;
  for (int64_t r = r0 + warp; r < r1; r += kIdWarps) {
    const float* row = res + r * lp;
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
    for (int c = tid; c < lp; c += kIdThreads) slot[4 + c] = myr >= 0 ? res[(int64_t)myr * lp + c] : 0.0f;
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
      float n = -1.0f;
      int r = -1, sl = -1;
      for (int c = lane; c < G; c += 32) {
        const float cn = __ldcg(slots + (int64_t)c * slot_sz);
        const int cr = __float_as_int(__ldcg(slots + (int64_t)c * slot_sz + 1));
        if (cr >= 0 && id_better(cn, cr, n, r)) { n = cn; r = cr; sl = c; }
      }
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
    for (int64_t r = r0 + warp; r < r1; r += kIdWarps) {
      float* row = res + r * lp;
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
  if (grid < 1 || l > kMaxL || lp > kMaxL) return cudaErrorInvalidValue;
  void* args[] = {&res, &m, &l, &lp, &coef, &piv, &cand, &bar, &status};
  return cudaLaunchCooperativeKernel((void*)id_pivot_kernel, dim3(grid), dim3(kIdThreads), args, 0, st);
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
