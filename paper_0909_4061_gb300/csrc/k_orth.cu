// Orthonormalisation of a tall sample matrix by Cholesky QR (Algorithm 4.1
// step 3; Section 4.1 asks for a stable orthonormaliser, and Cholesky QR
// repeated -- with a shifted first round for ill-conditioned samples --
// gives the same Q as Householder QR with diag(R) > 0 in exact arithmetic).
//
// One round on Y (rows x l, float32):
//   gram_partial  : G_b = Y_b^T Y_b over row blocks b (float32 FMA)
//   gram_reduce   : G = sum_b G_b in a fixed order with Kahan compensation
//   cholesky      : G + s I = R^T R in one CTA (s = l u tr(G) in a shifted
//                   round, else 0), pivots below l u max(diag G) replaced by
//                   that floor (rank-deficient samples), then R^-1 by
//                   column-oriented forward substitution
//   apply         : Q = Y R^-1 (the float32 GEMM of k_gemm_simt.cu)
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {
namespace {

constexpr int GT = 128;  // Gram tile edge handled by one CTA (256 threads x 8 x 8)
constexpr int GR = 32;   // rows staged in shared memory per step

__global__ void __launch_bounds__(256) gram_partial_kernel(const float* __restrict__ src, int splits,
                                                           int64_t split_stride,
                                                           float* __restrict__ y_out, int64_t rows,
                                                           int lp, float* __restrict__ gpart,
                                                           int64_t rows_per_blk) {
  extern __shared__ __align__(16) float ys[];  // [GR][lp]
  const int blk = blockIdx.x;
  // tile pair (I, J), I <= J, enumerated row by row
  int I = 0, J = blockIdx.y;
  {
    const int T = (lp + GT - 1) / GT;
    int idx = blockIdx.y;
    while (idx >= T - I) { idx -= T - I; ++I; }
    J = I + idx;
  }
  const int64_t r0 = (int64_t)blk * rows_per_blk;
  const int64_t r1 = min(rows, r0 + rows_per_blk);
  const int ti = threadIdx.x / 16, tj = threadIdx.x % 16;
  const int ib = I * GT + ti * 8, jb = J * GT + tj * 8;
  const bool write_y = (splits > 1) && (blockIdx.y == 0);

  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;

  const int lp4 = lp / 4;  // lp is a multiple of 16: whole float4 per row
  for (int64_t rb = r0; rb < r1; rb += GR) {
    const int nr = (int)min((int64_t)GR, r1 - rb);
    __syncthreads();
    for (int e = threadIdx.x; e < GR * lp4; e += blockDim.x) {
      const int rr = e / lp4, c4 = e - rr * lp4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (rr < nr) {
        const int64_t off = (rb + rr) * lp + 4 * c4;
        v = *reinterpret_cast<const float4*>(src + off);
        for (int s = 1; s < splits; ++s) {
          const float4 w = *reinterpret_cast<const float4*>(src + off + (int64_t)s * split_stride);
          v.x += w.x; v.y += w.y; v.z += w.z; v.w += w.w;
        }
        if (write_y) *reinterpret_cast<float4*>(y_out + off) = v;
      }
      *reinterpret_cast<float4*>(ys + rr * lp + 4 * c4) = v;
    }
    __syncthreads();
    for (int r = 0; r < nr; ++r) {
      float yi[8], yj[8];
      // lp is a multiple of 16 and ib, jb of 8: a row segment is in or out as a whole
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      const float4* pi = reinterpret_cast<const float4*>(ys + r * lp + ib);
      const float4* pj = reinterpret_cast<const float4*>(ys + r * lp + jb);
      const float4 i0 = ib < lp ? pi[0] : z4, i1 = ib < lp ? pi[1] : z4;
      const float4 j0 = jb < lp ? pj[0] : z4, j1 = jb < lp ? pj[1] : z4;
      yi[0] = i0.x; yi[1] = i0.y; yi[2] = i0.z; yi[3] = i0.w;
      yi[4] = i1.x; yi[5] = i1.y; yi[6] = i1.z; yi[7] = i1.w;
      yj[0] = j0.x; yj[1] = j0.y; yj[2] = j0.z; yj[3] = j0.w;
      yj[4] = j1.x; yj[5] = j1.y; yj[6] = j1.z; yj[7] = j1.w;
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(yi[a], yj[b], acc[a][b]);
    }
  }
  float* g = gpart + (int64_t)blk * lp * lp;
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int i = ib + a, j = jb + b;
      if (i < lp && j < lp) {
        g[(int64_t)i * lp + j] = acc[a][b];
        if (I != J) g[(int64_t)j * lp + i] = acc[a][b];
      }
    }
}

__global__ void gram_reduce_kernel(const float* __restrict__ gpart, int nblk, int lp,
                                   float* __restrict__ g) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)lp * lp;
  if (e >= n) return;
  float s = 0.0f, c = 0.0f;  // Kahan-compensated sum in a fixed order
  int b = 0;
  for (; b + 8 <= nblk; b += 8) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = gpart[(int64_t)(b + u) * n + e];   // loads in flight together
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float y = v[u] - c;
      const float t = s + y;
      c = (t - s) - y;
      s = t;
    }
  }
  for (; b < nblk; ++b) {
    const float y = gpart[(int64_t)b * n + e] - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  g[e] = s;
}

__device__ __forceinline__ int tri_off(int i) { return i * (i + 1) / 2; }            // row i of packed lower
__device__ __forceinline__ int col_off(int j, int l) { return j * l - j * (j - 1) / 2; }  // column j of packed lower (by columns)

__global__ void __launch_bounds__(1024) cholesky_kernel(const float* __restrict__ g, int l, int lp,
                                                        int shifted, float* __restrict__ lbuf,
                                                        float* __restrict__ r_out,
                                                        float* __restrict__ rinv,
                                                        float* __restrict__ racc, int racc_init,
                                                        uint32_t* status) {
  extern __shared__ __align__(16) float sm[];
  float* Lp = sm;                             // packed lower triangle, l (l + 1) / 2
  float* cvec = sm + tri_off(l) + 4;          // [kMaxL]
  __shared__ float s_red[2][32];
  __shared__ float s_shift, s_floor;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ntri = tri_off(l);  // l (l + 1) / 2 entries

  // 1. load the lower triangle, trace and largest diagonal entry
  for (int e = tid; e < ntri; e += nt) {
    int i = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
    while (tri_off(i + 1) <= e) ++i;
    while (tri_off(i) > e) --i;
    const int j = e - tri_off(i);
    Lp[e] = g[(int64_t)i * lp + j];
  }
  float tr = 0.0f, mx = 0.0f;
  bool bad = false;
  for (int i = tid; i < l; i += nt) {
    const float d = g[(int64_t)i * lp + i];
    if (!isfinite(d)) bad = true;
    tr += d;
    mx = fmaxf(mx, d);
  }
  if (bad) set_status(status, ST_NONFINITE);
  tr = warp_sum(tr);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((tid & 31) == 0) { s_red[0][tid >> 5] = tr; s_red[1][tid >> 5] = mx; }
  __syncthreads();
  if (tid == 0) {
    float t = 0.0f, m = 0.0f;
    for (int w = 0; w < (nt + 31) / 32; ++w) { t += s_red[0][w]; m = fmaxf(m, s_red[1][w]); }
    s_shift = shifted ? (float)l * kEpsF32 * t : 0.0f;
    s_floor = fmaxf((float)l * kEpsF32 * m, 1e-30f);
  }
  __syncthreads();
  const float shift = s_shift, pfloor = s_floor;
  for (int i = tid; i < l; i += nt) Lp[tri_off(i) + i] += shift;
  __syncthreads();

  // 2. right-looking Cholesky, column by column
  for (int j = 0; j < l; ++j) {
    float d = Lp[tri_off(j) + j];
    if (!(d > pfloor)) {
      if (tid == 0) set_status(status, isnan(d) ? ST_NONFINITE : ST_RANK_DEFICIENT);
      d = pfloor;
    }
    const float piv = sqrtf(d);
    const float rp = 1.0f / piv;
    for (int i = j + 1 + tid; i < l; i += nt) {
      const float v = Lp[tri_off(i) + j] * rp;
      cvec[i] = v;
      Lp[tri_off(i) + j] = v;
    }
    __syncthreads();
    if (tid == 0) Lp[tri_off(j) + j] = piv;
    const int s = l - j - 1;
    const int cnt = s * (s + 1) / 2;
    for (int e = tid; e < cnt; e += nt) {
      int a = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
      while ((a + 1) * (a + 2) / 2 <= e) ++a;
      while (a * (a + 1) / 2 > e) --a;
      const int b = e - a * (a + 1) / 2;
      const int i = j + 1 + a, k = j + 1 + b;
      Lp[tri_off(i) + k] -= cvec[i] * cvec[k];
    }
    __syncthreads();
  }

  // 3. R = L^T into r_out, L (row-major lower) into lbuf, zero padding
  for (int e = tid; e < lp * lp; e += nt) {
    const int a = e / lp, b = e % lp;  // r_out[a][b] = L[b][a] for b >= a
    r_out[e] = (a < l && b < l && b >= a) ? Lp[tri_off(b) + a] : 0.0f;
    lbuf[e] = (a < l && b < l && b <= a) ? Lp[tri_off(a) + b] : 0.0f;
  }
  __syncthreads();

  // 4. X = L^-1 (lower), column j by warp j mod 32, stored by columns in Lp's space
  float* Xc = Lp;
  const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  for (int j = warp; j < l; j += nw) {
    float* xj = Xc + col_off(j, l);  // xj[i - j] = X(i, j)
    const float djj = lbuf[(int64_t)j * lp + j];
    if (lane == 0) xj[0] = 1.0f / djj;
    __syncwarp();
    for (int i = j + 1; i < l; ++i) {
      const float* li = lbuf + (int64_t)i * lp;
      float part = 0.0f;
      for (int k = j + lane; k < i; k += 32) part = fmaf(li[k], xj[k - j], part);
      part = warp_sum(part);
      if (lane == 0) xj[i - j] = -part / li[i];
      __syncwarp();
    }
  }
  __syncthreads();

  // 5. R^-1 = X^T (upper)
  for (int e = tid; e < lp * lp; e += nt) {
    const int a = e / lp, b = e % lp;
    rinv[e] = (a < l && b < l && b >= a) ? Xc[col_off(a, l) + (b - a)] : 0.0f;
  }
  __syncthreads();

  // 6. accumulate the triangular factor across rounds: racc <- R racc
  if (racc) {
    float* tmp = Lp;  // packed upper by rows: (a, b), b >= a, at a*l - a(a-1)/2 + (b - a)
    for (int e = tid; e < ntri; e += nt) {
      // decode (a, b) of the packed-upper index e
      int a = 0, rem = e;
      while (rem >= l - a) { rem -= l - a; ++a; }
      const int b = a + rem;
      float v;
      if (racc_init) {
        v = r_out[(int64_t)a * lp + b];
      } else {
        v = 0.0f;
        for (int c = a; c <= b; ++c) v = fmaf(r_out[(int64_t)a * lp + c], racc[(int64_t)c * lp + b], v);
      }
      tmp[e] = v;
    }
    __syncthreads();
    for (int e = tid; e < lp * lp; e += nt) {
      const int a = e / lp, b = e % lp;
      racc[e] = (a < l && b < l && b >= a) ? tmp[a * l - a * (a - 1) / 2 + (b - a)] : 0.0f;
    }
  }
}

// Blocked Cholesky G + sI = L L^T and X = L^-1 in one CTA, both held in shared
// memory as full squares (row stride lp + 1), for lp <= 160.  The factor works on
// the padded size lp (a multiple of 16) with identity rows and columns beyond l,
// so every block is a full 16 x 16 and every inner loop has a compile-time trip
// count (unrolled, shared-memory loads in flight together).  Per block column:
// the diagonal block is factored and inverted by warp 0 in registers, the panel
// below it is L_iJ = A_iJ L_JJ^-T (a small product with the block inverse), and
// the trailing lower triangle is updated by all threads.  The off-diagonal blocks
// of the inverse follow block row by block row.  Outputs: R = L^T, R^-1 = X^T and
// the optional product racc <- R racc, restricted to l x l (zero elsewhere).
constexpr int CB = 16;

__global__ void __launch_bounds__(512) cholesky_blocked_kernel(
    const float* __restrict__ g, int l, int lp, int shifted, float* __restrict__ r_out,
    float* __restrict__ rinv, float* __restrict__ racc, int racc_init, uint32_t* status) {
  extern __shared__ __align__(16) float sm[];
  const int ld = lp + 1;
  float* A = sm;               // lower: L
  float* X = sm + lp * ld;     // lower: L^-1
  __shared__ float s_red[2][32];
  __shared__ float s_shift, s_floor;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  const int nb16 = lp / CB;

  // load the lower triangle of G (identity beyond l), clear X; rows by warps
  for (int i = warp; i < lp; i += nw) {
    const float* gi = g + (int64_t)i * lp;
    for (int j = lane; j < lp; j += 32) {
      float v = 0.0f;
      if (i < l && j < l) v = gi[j];
      else if (i == j) v = 1.0f;
      A[i * ld + j] = (j <= i) ? v : 0.0f;
      X[i * ld + j] = 0.0f;
    }
  }
  float tr = 0.0f, mx = 0.0f;
  bool bad = false;
  for (int i = tid; i < l; i += nt) {
    const float d = g[(int64_t)i * lp + i];
    if (!isfinite(d)) bad = true;
    tr += d;
    mx = fmaxf(mx, d);
  }
  if (bad) set_status(status, ST_NONFINITE);
  tr = warp_sum(tr);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) { s_red[0][warp] = tr; s_red[1][warp] = mx; }
  __syncthreads();
  if (tid == 0) {
    float t = 0.0f, m = 0.0f;
    for (int w = 0; w < nw; ++w) { t += s_red[0][w]; m = fmaxf(m, s_red[1][w]); }
    s_shift = shifted ? (float)l * kEpsF32 * t : 0.0f;
    s_floor = fmaxf((float)l * kEpsF32 * m, 1e-30f);
  }
  __syncthreads();
  const float pfloor = s_floor;
  for (int i = tid; i < l; i += nt) A[i * ld + i] += s_shift;
  __syncthreads();

  for (int jb = 0; jb < nb16; ++jb) {
    const int J = jb * CB;
    // (1) diagonal block by warp 0 in registers: lane i < 16 holds row i
    if (warp == 0) {
      float a[CB];
#pragma unroll
      for (int j = 0; j < CB; ++j)
        a[j] = (lane < CB) ? (j <= lane ? A[(J + lane) * ld + J + j] : 0.0f) : (j == lane ? 1.0f : 0.0f);
#pragma unroll
      for (int j = 0; j < CB; ++j) {
        float d = __shfl_sync(0xffffffffu, a[j], j);
        if (J + j < l && !(d > pfloor)) {
          if (lane == 0) set_status(status, isnan(d) ? ST_NONFINITE : ST_RANK_DEFICIENT);
          d = pfloor;
        }
        const float piv = sqrtf(d);
        const float rp = 1.0f / piv;
        const float lij = (lane == j) ? piv : (lane > j ? a[j] * rp : 0.0f);
        a[j] = lij;
#pragma unroll
        for (int k = j + 1; k < CB; ++k) {
          const float lkj = __shfl_sync(0xffffffffu, lij, k);
          if (lane >= k) a[k] = fmaf(-lij, lkj, a[k]);
        }
      }
      float x[CB];
#pragma unroll
      for (int i = 0; i < CB; ++i) {
        float v = 0.0f;
#pragma unroll
        for (int k = 0; k < i; ++k) {
          const float lik = __shfl_sync(0xffffffffu, a[k], i);
          if (k >= lane) v = fmaf(lik, x[k], v);
        }
        const float lii = __shfl_sync(0xffffffffu, a[i], i);
        x[i] = (i > lane) ? -v / lii : (i == lane ? 1.0f / lii : 0.0f);
      }
      if (lane < CB) {
#pragma unroll
        for (int j = 0; j < CB; ++j)
          if (j <= lane) A[(J + lane) * ld + J + j] = a[j];
#pragma unroll
        for (int i = 0; i < CB; ++i)
          if (i >= lane) X[(J + i) * ld + J + lane] = x[i];
      }
    }
    __syncthreads();
    // (2) panel: l_ij = sum_{k<=j} a_ik X_JJ(j, k), rows below the block; staged in the
    // strictly lower part of X (free until the inverse), then copied into A
    const int prow = lp - J - CB;
    for (int e = tid; e < prow * CB; e += nt) {
      const int i = J + CB + (e >> 4), j = e & (CB - 1);
      const float* ai = A + i * ld + J;
      const float* xj = X + (J + j) * ld + J;
      float v = 0.0f;
#pragma unroll
      for (int k = 0; k < CB; ++k) v = fmaf(ai[k], xj[k], v);   // X_JJ(j, k) = 0 for k > j
      X[i * ld + J + j] = v;
    }
    __syncthreads();
    for (int e = tid; e < prow * CB; e += nt) {
      const int i = J + CB + (e >> 4), j = e & (CB - 1);
      A[i * ld + J + j] = X[i * ld + J + j];
      X[i * ld + J + j] = 0.0f;
    }
    __syncthreads();
    // (3) trailing lower triangle: A_ik -= L_iJ . L_kJ  (16-term dots, unrolled)
    const int s0 = J + CB, sz = lp - s0;
    for (int e = tid; e < sz * sz; e += nt) {
      const int ii = e / sz, kk = e - ii * sz;
      if (kk > ii) continue;
      const int i = s0 + ii, k = s0 + kk;
      const float* li = A + i * ld + J;
      const float* lk = A + k * ld + J;
      float acc = 0.0f;
#pragma unroll
      for (int j = 0; j < CB; ++j) acc = fmaf(li[j], lk[j], acc);
      A[i * ld + k] -= acc;
    }
    __syncthreads();
  }

  // off-diagonal blocks of the inverse, block row Ib after block row Ib-1:
  // S(r, c) = sum_{c<=k<I} L(I+r, k) X(k, c) into A's free upper triangle, then
  // X(I+r, c) = -sum_{t<=r} X_II(r, t) S(t, c)
  for (int Ib = 1; Ib < nb16; ++Ib) {
    const int I = Ib * CB;
    for (int e = tid; e < CB * I; e += nt) {
      const int r = e / I, c = e - r * I;
      const float* lr = A + (I + r) * ld;
      float v = 0.0f;
      for (int kb = c / CB; kb < Ib; ++kb) {
        const int k0 = kb * CB;
#pragma unroll
        for (int kk = 0; kk < CB; ++kk) v = fmaf(lr[k0 + kk], X[(k0 + kk) * ld + c], v);
      }
      A[c * ld + I + r] = v;
    }
    __syncthreads();
    for (int e = tid; e < CB * I; e += nt) {
      const int r = e / I, c = e - r * I;
      const float* xr = X + (I + r) * ld + I;
      float v = 0.0f;
#pragma unroll
      for (int t2 = 0; t2 < CB; ++t2) v = fmaf(xr[t2], A[c * ld + I + t2], v);   // X_II(r, t) = 0, t > r
      X[(I + r) * ld + c] = -v;
    }
    __syncthreads();
  }

  // outputs: R = L^T, R^-1 = X^T restricted to l x l; rows by warps (no division)
  for (int a = warp; a < lp; a += nw) {
    for (int b = lane; b < lp; b += 32) {
      const bool up = (a < l && b < l && b >= a);
      r_out[(int64_t)a * lp + b] = up ? A[b * ld + a] : 0.0f;
      rinv[(int64_t)a * lp + b] = up ? X[b * ld + a] : 0.0f;
    }
  }
  if (racc) {
    __syncthreads();
    float* Pm = X;   // racc <- R racc, into the free X space
    for (int a = warp; a < l; a += nw) {
      for (int b = lane; b < l; b += 32) {
        float v = 0.0f;
        if (b >= a) {
          if (racc_init) {
            v = A[b * ld + a];
          } else {
            for (int c = a; c <= b; ++c) v = fmaf(A[c * ld + a], racc[(int64_t)c * lp + b], v);
          }
        }
        Pm[a * ld + b] = v;
      }
    }
    __syncthreads();
    for (int a = warp; a < lp; a += nw)
      for (int b = lane; b < lp; b += 32)
        racc[(int64_t)a * lp + b] = (a < l && b < l && b >= a) ? Pm[a * ld + b] : 0.0f;
  }
}

__global__ void to_bf16_t_kernel(const float* __restrict__ x, int64_t rows, int lp,
                                 __nv_bfloat16* __restrict__ out, int64_t ld_t, int split,
                                 int lo_off) {
  __shared__ float tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int i = ty; i < 32; i += 8) {
    const int64_t r = r0 + i;
    const int c = c0 + tx;
    tile[i][tx] = (r < rows && c < lp) ? x[r * lp + c] : 0.0f;
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int c = c0 + i;
    const int64_t r = r0 + tx;
    if (c < lp && r < rows) {
      const float v = tile[tx][i];
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      out[(int64_t)c * ld_t + r] = hi;
      if (split) out[(int64_t)(lo_off + c) * ld_t + r] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
  }
}

__global__ void split_bf16_kernel(const float* __restrict__ x, int64_t rows, int64_t cols,
                                  int64_t ld, __nv_bfloat16* __restrict__ out, int64_t ld_out,
                                  int with_lo) {
  const int64_t n = rows * cols;
  const int64_t lo_off = rows * ld_out;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    const float v = x[r * ld + c];
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    out[r * ld_out + c] = hi;
    if (with_lo) out[lo_off + r * ld_out + c] = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
}

__global__ void f32_to_bf16_kernel(const float* __restrict__ x, int64_t rows, int64_t cols,
                                   int64_t ld, __nv_bfloat16* __restrict__ out, int64_t ld_out) {
  const int64_t n = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    out[r * ld_out + c] = __float2bfloat16_rn(x[r * ld + c]);
  }
}

__global__ void gather_kernel(const float* __restrict__ src, int splits, int64_t split_stride,
                              int64_t lds, float* __restrict__ dst, int64_t ldd, int64_t rows,
                              int cols, int cols_pad) {
  const int64_t n = rows * cols_pad;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols_pad;
    const int c = (int)(e % cols_pad);
    float v = 0.0f;
    if (c < cols)
      for (int s = 0; s < splits; ++s) v += src[(int64_t)s * split_stride + r * lds + c];
    dst[r * ldd + c] = v;
  }
}

}  // namespace

// Shared-memory limits of the one-CTA factorisation kernels, for every size they accept;
// set once per device (at plan creation) so no launch needs a host-side attribute call.
cudaError_t prepare_orth() {
  cudaError_t e = cudaFuncSetAttribute(cholesky_blocked_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)((size_t)2 * 160 * 161 * sizeof(float)));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(cholesky_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(((size_t)kMaxL * (kMaxL + 1) / 2 + kMaxL + 4 + kMaxL) *
                                    sizeof(float)));
}

int gram_blocks(int64_t rows) {
  const int64_t b = cdiv(rows, 64);
  return (int)(b < 4 * kNumSMs ? (b < 1 ? 1 : b) : 4 * kNumSMs);
}

cudaError_t launch_gram_partial(const float* src, int splits, int64_t split_stride, float* y_out,
                                int64_t rows, int lp, float* gpart, int nblk, cudaStream_t st) {
  const int T = (lp + GT - 1) / GT;
  const int npair = T * (T + 1) / 2;
  const int64_t rpb = round_up(cdiv(rows, nblk), GR);
  const size_t smem = (size_t)GR * lp * sizeof(float);  // <= 32 KB for lp <= 256
  gram_partial_kernel<<<dim3(nblk, npair), 256, smem, st>>>(src, splits, split_stride, y_out, rows,
                                                            lp, gpart, rpb);
  return cudaGetLastError();
}

cudaError_t launch_gram_reduce(const float* gpart, int nblk, int lp, float* g, cudaStream_t st) {
  const int64_t n = (int64_t)lp * lp;
  gram_reduce_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(gpart, nblk, lp, g);
  return cudaGetLastError();
}

cudaError_t launch_cholesky(const float* g, int l, int lp, int shifted, float* lbuf, float* r_out,
                            float* rinv, float* racc, int racc_init, uint32_t* status,
                            cudaStream_t st) {
  if (lp <= 160) {
    const size_t sm = (size_t)2 * lp * (lp + 1) * sizeof(float);
    cholesky_blocked_kernel<<<1, 512, sm, st>>>(g, l, lp, shifted, r_out, rinv, racc, racc_init,
                                                status);
    return cudaGetLastError();
  }
  const size_t smem = ((size_t)l * (l + 1) / 2 + l + 4 + kMaxL) * sizeof(float);
  cholesky_kernel<<<1, 1024, smem, st>>>(g, l, lp, shifted, lbuf, r_out, rinv, racc, racc_init,
                                         status);
  return cudaGetLastError();
}

cudaError_t launch_to_bf16_t(const float* x, int64_t rows, int lp, __nv_bfloat16* out, int64_t ld_t,
                             int split, int lo_off, cudaStream_t st) {
  const dim3 grid((unsigned)cdiv(rows, 32), (unsigned)cdiv(lp, 32));
  to_bf16_t_kernel<<<grid, dim3(32, 8), 0, st>>>(x, rows, lp, out, ld_t, split, lo_off);
  return cudaGetLastError();
}

cudaError_t launch_split_bf16(const float* x, int64_t rows, int64_t cols, int64_t ld,
                              __nv_bfloat16* out, int64_t ld_out, int with_lo, cudaStream_t st) {
  const int64_t n = rows * cols;
  if (n == 0) return cudaSuccess;
  const unsigned grid = (unsigned)(cdiv(n, 256) < 16 * kNumSMs ? cdiv(n, 256) : 16 * kNumSMs);
  split_bf16_kernel<<<grid, 256, 0, st>>>(x, rows, cols, ld, out, ld_out, with_lo);
  return cudaGetLastError();
}

cudaError_t launch_f32_to_bf16(const float* x, int64_t rows, int64_t cols, int64_t ld,
                               __nv_bfloat16* out, int64_t ld_out, cudaStream_t st) {
  const int64_t n = rows * cols;
  const unsigned grid = (unsigned)(cdiv(n, 256) < 4 * 8 * kNumSMs ? cdiv(n, 256) : 4 * 8 * kNumSMs);
  f32_to_bf16_kernel<<<grid, 256, 0, st>>>(x, rows, cols, ld, out, ld_out);
  return cudaGetLastError();
}

cudaError_t launch_gather(const float* src, int splits, int64_t split_stride, int64_t lds,
                          float* dst, int64_t ldd, int64_t rows, int cols, int cols_pad,
                          cudaStream_t st) {
  const int64_t n = rows * cols_pad;
  if (n == 0) return cudaSuccess;
  const unsigned grid = (unsigned)(cdiv(n, 256) < 8 * kNumSMs ? cdiv(n, 256) : 8 * kNumSMs);
  gather_kernel<<<grid, 256, 0, st>>>(src, splits, split_stride, lds, dst, ldd, rows, cols,
                                      cols_pad);
  return cudaGetLastError();
}

}  // namespace rsvd
