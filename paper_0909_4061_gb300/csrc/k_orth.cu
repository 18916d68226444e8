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
//                   that floor and the column below them set to zero
//                   (rank-deficient samples), then R^-1 by forward substitution
//   apply         : Q = Y R^-1 (the float32 GEMM of k_gemm_simt.cu; fused with
//                   the next Gram for l_p <= 128)
// Wider samples (l_p > 128) form the Gram partials on the tensor cores (k_gram_tc.cu).
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
  // partial block (row-major lp x lp); rows ib..ib+7 as two float4 per row, so a
  // warp writes two 512-byte row segments (the mirrored tile of an off-diagonal pair
  // goes out column by column)
  float* g = gpart + (int64_t)blk * lp * lp;
  if (ib < lp && jb < lp) {
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      float4* dst = reinterpret_cast<float4*>(g + (int64_t)(ib + a) * lp + jb);
      dst[0] = make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
      dst[1] = make_float4(acc[a][4], acc[a][5], acc[a][6], acc[a][7]);
    }
    if (I != J) {
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        float4* dst = reinterpret_cast<float4*>(g + (int64_t)(jb + b) * lp + ib);
        dst[0] = make_float4(acc[0][b], acc[1][b], acc[2][b], acc[3][b]);
        dst[1] = make_float4(acc[4][b], acc[5][b], acc[6][b], acc[7][b]);
      }
    }
  }
}

// G = sum_b G_b for the lower triangle (the factorisation reads no more): a block
// of 512 threads takes 32 consecutive elements (one per lane) and splits the nblk
// partials into 16 contiguous ranges (one per warp), each summed with Kahan
// compensation with all of its loads in flight; the 16 (sum, compensation) pairs
// are then combined in range order, so the result does not depend on timing.
constexpr int kRedSplit = 16;
constexpr int kRedBatch = 24;

// One Cholesky-QR step fused with the Gram matrix of the next, for l_p <= 128 (APPLY), and
// the Gram matrix of a sample alone (!APPLY), both on 64-row tiles of Y.
//
// Apply: Q = Y R^-1 with R^-1 upper triangular, so column block c (8 columns) of Q needs
// only rows 0 .. 8c + 7 of R^-1.  Warp w owns the column blocks w and NCB - 1 - w, which
// makes every warp's share of the triangle the same (NCB + 1 blocks of 8 products), and
// each lane owns two rows of the tile.  The tile of Y sits transposed in shared memory
// (one 8-byte load gives a lane its two rows of a column) and R^-1 row-major (the 8
// columns of a block are one broadcast read per warp).
// Gram: only the lower triangle is formed (the factorisation reads no more), as 8 x 4
// (or 8 x 8) tiles of Q^T Q over the tile's rows, one tile per thread, accumulated over
// the CTA's row tiles and written as this CTA's partial for the reduce kernel.
// Products are paired into fma.rn.f32x2, which rounds each lane exactly as fmaf does: the
// sums, and their order over rows and columns, are those of the plain definition.
constexpr int TR_ROWS = 64;
constexpr int TR_LDT = TR_ROWS + 2;   // transposed tile stride: conflict-free staging stores

template <int LP, bool APPLY>
struct TriCfg {
  static constexpr int NCB = LP / 8;                 // column blocks of 8 (even)
  static constexpr int NP = NCB / 2;                 // warps: one block pair each
  static constexpr int T = 32 * NP;
  static constexpr int LDQ = LP + 4;
  static constexpr int NB8 = NCB * (NCB + 1) / 2;    // 8 x 8 blocks of the lower triangle
  static constexpr int TW = (2 * NB8 <= T) ? 4 : 8;  // Gram tile width
  static constexpr int NTASK = NB8 * (8 / TW);
  static constexpr int UFL = APPLY ? (LP * TR_LDT > TR_ROWS * LDQ ? LP * TR_LDT : TR_ROWS * LDQ)
                                   : TR_ROWS * LDQ;
  static constexpr int SMEM = (APPLY ? LP * LDQ + UFL : UFL) * (int)sizeof(float);
};

// 16-byte global -> shared copy that does not pass through registers (L2 only), so a
// thread can have all of its copies in flight at once.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

typedef unsigned long long f2_t;   // two float32 values, the first in the low half
__device__ __forceinline__ f2_t pk2(float a, float b) {
  f2_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 upk2(f2_t v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ void fma2(f2_t& acc, f2_t a, f2_t b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}

template <int LP, bool APPLY>
__global__ void __launch_bounds__(TriCfg<LP, APPLY>::T, (LP >= 128 ? 1 : 2))
    orth_tri_kernel(const float* __restrict__ y, int splits, int64_t split_stride,
                    float* __restrict__ q, int64_t rows, const float* __restrict__ rinv,
                    float* __restrict__ gpart, int64_t rows_per_blk, int do_gram) {
  using C = TriCfg<LP, APPLY>;
  constexpr int NCB = C::NCB, NP = C::NP, T = C::T, LDQ = C::LDQ, TW = C::TW;
  constexpr int NC4 = LP / 4;
  extern __shared__ __align__(16) float sm[];
  float* Rs = sm;                                 // R^-1, LP x LDQ (APPLY)
  float* Ub = sm + (APPLY ? LP * LDQ : 0);        // Y^T (LP x TR_LDT), then Q (TR_ROWS x LDQ)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_blk, r1 = min(rows, r0 + rows_per_blk);
  // With APPLY, Y comes from the Cholesky-QR round before the factorisation this launch
  // depends on (two or more launches back): the first tile's loads go out before the wait.
  float4 vpre[8];
  if (APPLY) {
    const int nr0 = (int)min((int64_t)TR_ROWS, r1 - r0);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int s = warp + NP * k, rg = s & 7, cg = s >> 3;
      const int r = 8 * rg + (lane & 7), c4 = 4 * cg + (lane >> 3);
      vpre[k] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < nr0) vpre[k] = *reinterpret_cast<const float4*>(y + (r0 + r) * LP + 4 * c4);
    }
  }
  pdl_wait();
  pdl_trigger();
  if (APPLY) {   // R^-1 into shared memory, waited for with the first tile of Y
    for (int e = tid; e < LP * NC4; e += T) {
      const int r = e / NC4, c4 = e - r * NC4;
      cp_async16(Rs + r * LDQ + 4 * c4, rinv + r * LP + 4 * c4);
    }
  }
  // this thread's Gram tile: rows 8 ga .. 8 ga + 7, columns gc .. gc + TW - 1 (gc <= 8 ga)
  const bool has_task = tid < C::NTASK;
  int ga = 0, gc = 0;
  {
    int t = has_task ? tid : 0;
    while (t >= (ga + 1) * (8 / TW)) { t -= (ga + 1) * (8 / TW); ++ga; }
    gc = TW * t;
  }
  f2_t g[4][TW];   // g[p][c] = (G(8 ga + 2p, gc + c), G(8 ga + 2p + 1, gc + c))
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int c = 0; c < TW; ++c) g[p][c] = 0ull;
  const int cb0 = warp, cb1 = NCB - 1 - warp;
  for (int64_t rb = r0; rb < r1; rb += TR_ROWS) {
    const int nr = (int)min((int64_t)TR_ROWS, r1 - rb);
    __syncthreads();   // the previous tile is no longer read
    if (APPLY) {
      // stage Y^T: per step a warp takes 8 rows x 4 float4 columns (lane = 8 cc + rr), so
      // the global reads are whole sectors and the transposed stores hit 32 banks
      {
        float4 v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int s = warp + NP * k, rg = s & 7, cg = s >> 3;
          const int r = 8 * rg + (lane & 7), c4 = 4 * cg + (lane >> 3);
          v[k] = vpre[k];
          if (rb != r0) {
            v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < nr) v[k] = *reinterpret_cast<const float4*>(y + (rb + r) * LP + 4 * c4);
          }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int s = warp + NP * k, rg = s & 7, cg = s >> 3;
          const int r = 8 * rg + (lane & 7), c4 = 4 * cg + (lane >> 3);
          float* d = Ub + (4 * c4) * TR_LDT + r;
          d[0] = v[k].x; d[TR_LDT] = v[k].y; d[2 * TR_LDT] = v[k].z; d[3 * TR_LDT] = v[k].w;
        }
      }
      cp_async_wait_all();
      __syncthreads();
      f2_t a0[2][4], a1[2][4];   // rows 2 lane + rr; column pairs of blocks cb0, cb1
#pragma unroll
      for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int c = 0; c < 4; ++c) { a0[rr][c] = 0ull; a1[rr][c] = 0ull; }
      const float* yt = Ub + 2 * lane;
      const float* p0 = Rs + 8 * cb0;
      const float* p1 = Rs + 8 * cb1;
      const int k0 = 8 * (cb0 + 1), k1 = 8 * (cb1 + 1);
      int i = 0;
#pragma unroll 2
      for (; i < k0; ++i) {
        const float2 yv = *reinterpret_cast<const float2*>(yt + i * TR_LDT);
        const f2_t y0 = pk2(yv.x, yv.x), y1 = pk2(yv.y, yv.y);
        const ulonglong2 x0 = *reinterpret_cast<const ulonglong2*>(p0 + i * LDQ);
        const ulonglong2 x1 = *reinterpret_cast<const ulonglong2*>(p0 + i * LDQ + 4);
        const ulonglong2 z0 = *reinterpret_cast<const ulonglong2*>(p1 + i * LDQ);
        const ulonglong2 z1 = *reinterpret_cast<const ulonglong2*>(p1 + i * LDQ + 4);
        fma2(a0[0][0], y0, x0.x); fma2(a0[0][1], y0, x0.y); fma2(a0[0][2], y0, x1.x); fma2(a0[0][3], y0, x1.y);
        fma2(a0[1][0], y1, x0.x); fma2(a0[1][1], y1, x0.y); fma2(a0[1][2], y1, x1.x); fma2(a0[1][3], y1, x1.y);
        fma2(a1[0][0], y0, z0.x); fma2(a1[0][1], y0, z0.y); fma2(a1[0][2], y0, z1.x); fma2(a1[0][3], y0, z1.y);
        fma2(a1[1][0], y1, z0.x); fma2(a1[1][1], y1, z0.y); fma2(a1[1][2], y1, z1.x); fma2(a1[1][3], y1, z1.y);
      }
#pragma unroll 2
      for (; i < k1; ++i) {
        const float2 yv = *reinterpret_cast<const float2*>(yt + i * TR_LDT);
        const f2_t y0 = pk2(yv.x, yv.x), y1 = pk2(yv.y, yv.y);
        const ulonglong2 z0 = *reinterpret_cast<const ulonglong2*>(p1 + i * LDQ);
        const ulonglong2 z1 = *reinterpret_cast<const ulonglong2*>(p1 + i * LDQ + 4);
        fma2(a1[0][0], y0, z0.x); fma2(a1[0][1], y0, z0.y); fma2(a1[0][2], y0, z1.x); fma2(a1[0][3], y0, z1.y);
        fma2(a1[1][0], y1, z0.x); fma2(a1[1][1], y1, z0.y); fma2(a1[1][2], y1, z1.x); fma2(a1[1][3], y1, z1.y);
      }
      __syncthreads();   // every warp has read Y^T before Q overwrites it
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const int row = 2 * lane + rr;
        const float2 u0 = upk2(a0[rr][0]), u1 = upk2(a0[rr][1]), u2 = upk2(a0[rr][2]), u3 = upk2(a0[rr][3]);
        const float2 w0 = upk2(a1[rr][0]), w1 = upk2(a1[rr][1]), w2 = upk2(a1[rr][2]), w3 = upk2(a1[rr][3]);
        const float4 qa0 = make_float4(u0.x, u0.y, u1.x, u1.y), qa1 = make_float4(u2.x, u2.y, u3.x, u3.y);
        const float4 qb0 = make_float4(w0.x, w0.y, w1.x, w1.y), qb1 = make_float4(w2.x, w2.y, w3.x, w3.y);
        float* srow = Ub + row * LDQ;
        *reinterpret_cast<float4*>(srow + 8 * cb0) = qa0;
        *reinterpret_cast<float4*>(srow + 8 * cb0 + 4) = qa1;
        *reinterpret_cast<float4*>(srow + 8 * cb1) = qb0;
        *reinterpret_cast<float4*>(srow + 8 * cb1 + 4) = qb1;
        if (row < nr) {
          float* grow = q + (rb + row) * LP;
          *reinterpret_cast<float4*>(grow + 8 * cb0) = qa0;
          *reinterpret_cast<float4*>(grow + 8 * cb0 + 4) = qa1;
          *reinterpret_cast<float4*>(grow + 8 * cb1) = qb0;
          *reinterpret_cast<float4*>(grow + 8 * cb1 + 4) = qb1;
        }
      }
    } else if (splits == 1 && q == nullptr) {
      // stage Y row-major, every copy in flight; rows past the end are zero
      for (int e = tid; e < TR_ROWS * NC4; e += T) {
        const int r = e / NC4, c4 = e - r * NC4;
        if (r < nr) cp_async16(Ub + r * LDQ + 4 * c4, y + (rb + r) * LP + 4 * c4);
        else *reinterpret_cast<float4*>(Ub + r * LDQ + 4 * c4) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      cp_async_wait_all();
    } else {
      // stage Y row-major (the sum of the partial slabs), writing the sum out when asked
      for (int e = tid; e < TR_ROWS * NC4; e += T) {
        const int r = e / NC4, c4 = e - r * NC4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < nr) {
          const int64_t off = (rb + r) * LP + 4 * c4;
          v = *reinterpret_cast<const float4*>(y + off);
          for (int s = 1; s < splits; ++s) {
            const float4 w = *reinterpret_cast<const float4*>(y + off + (int64_t)s * split_stride);
            v.x += w.x; v.y += w.y; v.z += w.z; v.w += w.w;
          }
          if (q) *reinterpret_cast<float4*>(q + off) = v;
        }
        *reinterpret_cast<float4*>(Ub + r * LDQ + 4 * c4) = v;
      }
    }
    if (!do_gram) continue;
    __syncthreads();
    if (has_task) {
      const float* qa = Ub + 8 * ga;
      const float* qb = Ub + gc;
#pragma unroll 4
      for (int r = 0; r < nr; ++r) {
        const ulonglong2 i0 = *reinterpret_cast<const ulonglong2*>(qa + r * LDQ);
        const ulonglong2 i1 = *reinterpret_cast<const ulonglong2*>(qa + r * LDQ + 4);
        const f2_t ip[4] = {i0.x, i0.y, i1.x, i1.y};
        float jv[TW];
        {
          const float4 j0 = *reinterpret_cast<const float4*>(qb + r * LDQ);
          jv[0] = j0.x; jv[1] = j0.y; jv[2] = j0.z; jv[3] = j0.w;
          if constexpr (TW == 8) {
            const float4 j1 = *reinterpret_cast<const float4*>(qb + r * LDQ + 4);
            jv[4] = j1.x; jv[5] = j1.y; jv[6] = j1.z; jv[7] = j1.w;
          }
        }
#pragma unroll
        for (int c = 0; c < TW; ++c) {
          const f2_t jj = pk2(jv[c], jv[c]);
#pragma unroll
          for (int p = 0; p < 4; ++p) fma2(g[p][c], ip[p], jj);
        }
      }
    }
  }
  if (do_gram && has_task) {
    float* gp = gpart + (int64_t)blockIdx.x * LP * LP;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      float lo[TW], hi[TW];
#pragma unroll
      for (int c = 0; c < TW; ++c) {
        const float2 v = upk2(g[p][c]);
        lo[c] = v.x;
        hi[c] = v.y;
      }
      float* d0 = gp + (8 * ga + 2 * p) * LP + gc;
      float* d1 = d0 + LP;
#pragma unroll
      for (int c = 0; c < TW; c += 4) {
        *reinterpret_cast<float4*>(d0 + c) = make_float4(lo[c], lo[c + 1], lo[c + 2], lo[c + 3]);
        *reinterpret_cast<float4*>(d1 + c) = make_float4(hi[c], hi[c + 1], hi[c + 2], hi[c + 3]);
      }
    }
  }
}

__global__ void __launch_bounds__(512) gram_reduce_kernel(const float* __restrict__ gpart, int nblk,
                                                          int lp, float* __restrict__ g) {
  __shared__ float s_sum[kRedSplit][32], s_cmp[kRedSplit][32];
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t n = (int64_t)lp * lp;
  const int64_t e = (int64_t)blockIdx.x * 32 + lane;
  const int i = (int)(e / lp), j = (int)(e - (int64_t)i * lp);
  const bool live = e < n && j <= i;
  const int per = (nblk + kRedSplit - 1) / kRedSplit;
  const int b0 = w * per, b1 = min(nblk, b0 + per);
  float s = 0.0f, c = 0.0f;
  if (live) {
    for (int b = b0; b < b1; b += kRedBatch) {
      float v[kRedBatch];
#pragma unroll
      for (int u = 0; u < kRedBatch; ++u) v[u] = (b + u < b1) ? gpart[(int64_t)(b + u) * n + e] : 0.0f;
#pragma unroll
      for (int u = 0; u < kRedBatch; ++u) {
        const float y = v[u] - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
      }
    }
  }
  s_sum[w][lane] = s;
  s_cmp[w][lane] = c;
  __syncthreads();
  if (w == 0 && e < n) {
    float S = 0.0f, C = 0.0f;
    for (int q = 0; q < kRedSplit; ++q) {
      const float y = s_sum[q][lane] - (s_cmp[q][lane] + C);
      const float t = S + y;
      C = (t - S) - y;
      S = t;
    }
    g[e] = live ? S : 0.0f;
  }
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
    const bool low = !(d > pfloor);
    if (low) {
      if (tid == 0) set_status(status, isnan(d) ? ST_NONFINITE : ST_RANK_DEFICIENT);
      d = pfloor;
    }
    const float piv = sqrtf(d);
    // below a floored pivot the column is rounding noise (|a_ij| <= sqrt(a_ii a_jj) for a
    // semidefinite matrix): it is set to zero rather than scaled by 1 / sqrt(floor), which
    // would feed that noise, enlarged, into every later pivot
    const float cs = low ? 0.0f : 1.0f / piv;
    for (int i = j + 1 + tid; i < l; i += nt) {
      const float v = Lp[tri_off(i) + j] * cs;
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

// Blocked Cholesky G + sI = L L^T and X = L^-1 in one CTA of 512 threads, for
// LP = 16 NB <= 256: up to LP = 160 both held in shared memory as full squares; above,
// L in a padded row-packed form (143 KB at LP = 256) and X in global memory (L2).  The row stride
// LP + 4 keeps rows 16-byte aligned (float4 loads along a row) with an odd number of
// float4 per row (a column of float4 loads hits distinct banks).  The factor works
// on the padded size LP with identity rows and columns beyond l, so every block is
// a full 16 x 16.  Per block column J: warp 0 factors the diagonal block in registers
// (lane = row, the pivot column by shuffles, pivots by a Newton-refined reciprocal square
// root; entries above the diagonal collect scratch until their pivot zeroes them) and
// another warp inverts it; the panel below is L_iJ = A_iJ L_JJ^-T by forward
// substitution; the trailing lower triangle is updated by all warps, two rows per warp
// and one column per lane.  The off-diagonal blocks of
// X follow block row by block row: S = L_I,<I X_<I,<I in 2 x 4 register tiles, then
// X_I,<I = -X_II S.  Every inner product reads shared memory as float4, so the
// shared-memory pipe, not the FMA units, sets the pace only where unavoidable.
// Outputs: R = L^T, R^-1 = X^T and the optional product racc <- R racc, restricted
// to l x l.  The block loops stay rolled: unrolled, the code outgrows the
// instruction cache.
constexpr int CB = 16;

// Offset of row i in the padded row-packed form of a lower-triangular L (16-row block
// rows; row i holds 16 (i / 16 + 1) columns plus 4 floats of skew).
__host__ __device__ constexpr int pk_off(int i) {
  return 128 * (i / CB) * (i / CB + 1) + 64 * (i / CB) + (i % CB) * (16 * (i / CB) + 20);
}

__device__ __forceinline__ float dot4(const float4 a, const float4 b, float acc) {
  acc = fmaf(a.x, b.x, acc);
  acc = fmaf(a.y, b.y, acc);
  acc = fmaf(a.z, b.z, acc);
  return fmaf(a.w, b.w, acc);
}

__device__ __forceinline__ float4 axpy4(float s, const float4 x, float4 y) {
  y.x = fmaf(s, x.x, y.x);
  y.y = fmaf(s, x.y, y.y);
  y.z = fmaf(s, x.z, y.z);
  y.w = fmaf(s, x.w, y.w);
  return y;
}

template <int NB>
__global__ void __launch_bounds__(512, 1) cholesky_blocked_kernel(
    const float* __restrict__ g, int l, int shifted, float* __restrict__ r_out,
    float* __restrict__ rinv, float* __restrict__ racc, int racc_init, uint32_t* status,
    float* __restrict__ xg) {
  constexpr int LP = CB * NB;
  constexpr int LD = LP + 4;
  constexpr bool PACKED = NB > 10;       // L in padded row-packed form, L^-1 in global memory
  constexpr int NW = 16;                 // warps
  constexpr int NCOL = (LP + 31) / 32;   // columns per lane in row-by-warp loops
  constexpr int RCH = PACKED ? 4 : NB;   // rows per warp loaded together
  extern __shared__ __align__(16) float sm[];
  // Square form: A (L, scratch above the diagonal) and X = L^-1 as LP x LD squares; the
  // block-row products S of the inverse live in A's scratch upper triangle.
  // Packed form: row i of L holds columns 0 .. 16 (i / 16 + 1) - 1 (the diagonal block's
  // scratch included) plus 4 floats of skew, so float4 rows stay aligned and consecutive
  // rows fall in different banks; X lives in global memory (xg, LP x LP) and S in a
  // separate 16 x (LP + 4) block.
  float* A = sm;
  float* X = PACKED ? xg : sm + LP * LD;
  float* Sb = sm + pk_off(LP);   // packed form only
  auto arow = [&](int i) -> float* {
    return PACKED ? A + pk_off(i) : A + i * LD;
  };
  auto xrow = [&](int i) -> float* { return PACKED ? X + i * LP : X + i * LD; };
  auto alen = [&](int i) -> int { return PACKED ? CB * (i / CB + 1) : LP; };
  __shared__ float s_red[2][NW];
  __shared__ __align__(16) float s_lt[CB][CB];   // L_JJ^T of the latest diagonal block
  __shared__ __align__(16) float s_rpv[LP];      // 1 / L(j, j)
  __shared__ __align__(16) float s_csv[LP];      // scale of column j below the pivot (0 if floored)
  __shared__ float s_shift, s_floor;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;

  pdl_wait();
  pdl_trigger();
  // load the lower triangle of G (identity beyond l), all loads in flight together
  float tr = 0.0f, mx = 0.0f;
  bool bad = false;
#pragma unroll 1
  for (int r0 = 0; r0 < NB; r0 += RCH) {
    float v[RCH][NCOL];
#pragma unroll
    for (int r = 0; r < RCH; ++r)
#pragma unroll
      for (int c = 0; c < NCOL; ++c) {
        const int i = warp + NW * (r0 + r), j = lane + 32 * c;
        v[r][c] = (j <= i && i < l) ? g[i * LP + j] : 0.0f;   // lower triangle only
      }
#pragma unroll
    for (int r = 0; r < RCH; ++r)
#pragma unroll
      for (int c = 0; c < NCOL; ++c) {
        const int i = warp + NW * (r0 + r), j = lane + 32 * c;
        if (i < LP && j < LP) {   // the last group of RCH row blocks may run past LP
          float w = v[r][c];
          if (i == j) {
            if (i < l) {
              bad |= !isfinite(w);
              tr += w;
              mx = fmaxf(mx, w);
            } else {
              w = 1.0f;
            }
          }
          if (j < alen(i)) arow(i)[j] = (j <= i) ? w : 0.0f;
          xrow(i)[j] = 0.0f;
        }
      }
  }
  if (bad) set_status(status, ST_NONFINITE);
  tr = warp_sum(tr);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) { s_red[0][warp] = tr; s_red[1][warp] = mx; }
  __syncthreads();
  if (tid == 0) {
    float t = 0.0f, m = 0.0f;
    for (int w = 0; w < NW; ++w) { t += s_red[0][w]; m = fmaxf(m, s_red[1][w]); }
    s_shift = shifted ? (float)l * kEpsF32 * t : 0.0f;
    s_floor = fmaxf((float)l * kEpsF32 * m, 1e-30f);
  }
  __syncthreads();
  const float pfloor = s_floor;
  if (tid < l) arow(tid)[tid] += s_shift;
  __syncthreads();

  // Diagonal block J (16 x 16) by warp 0, lane r (and r + 16, which repeats it) holding row
  // r: per pivot j the pivot comes by a shuffle from lane j, every lane forms 1/sqrt of it
  // (hardware estimate and one Newton step y <- y (3 - d y^2) / 2), scales its entry of
  // column j and updates its row with the column's entries fetched by shuffles.  Entries
  // above the diagonal collect scratch until their own pivot zeroes them.  A pivot at or
  // below the floor is replaced by it and the column below it set to zero (a rank-deficient
  // sample); the first such pivot is reported.  Row r of L_JJ goes to A, its transpose to
  // s_lt, the reciprocal pivots to s_rpv and the column scales to s_csv.
  bool any_low = false;
  float dlow = 0.0f;
  auto diag_factor = [&](int J) {
    const int r = lane & 15;
    float a[CB];
    {
      const float4* src = reinterpret_cast<const float4*>(arow(J + r) + J);
#pragma unroll
      for (int q = 0; q < CB / 4; ++q) {
        const float4 t = src[q];
        a[4 * q] = t.x; a[4 * q + 1] = t.y; a[4 * q + 2] = t.z; a[4 * q + 3] = t.w;
      }
    }
    float myrp = 0.0f, mycs = 0.0f;
#pragma unroll
    for (int j = 0; j < CB; ++j) {
      float d = __shfl_sync(0xffffffffu, a[j], j, 16);
      const bool low = J + j < l && !(d > pfloor);   // the same in every lane
      if (low && !any_low) dlow = d;
      any_low |= low;
      d = low ? pfloor : d;
      float rp = rsqrtf(d);
      rp = rp * fmaf(-0.5f * d * rp, rp, 1.5f);
      const float cs = low ? 0.0f : rp;
      if (r == j) {
        myrp = rp;
        mycs = cs;
      }
      const float lij = (r == j) ? d * rp : (r > j ? a[j] * cs : 0.0f);
      a[j] = lij;
#pragma unroll
      for (int k = j + 1; k < CB; ++k) a[k] = fmaf(-lij, __shfl_sync(0xffffffffu, lij, k, 16), a[k]);
    }
    if (any_low && lane == 0) set_status(status, isnan(dlow) ? ST_NONFINITE : ST_RANK_DEFICIENT);
    if (lane < CB) {
      float4* dst = reinterpret_cast<float4*>(arow(J + r) + J);
#pragma unroll
      for (int q = 0; q < CB / 4; ++q) dst[q] = make_float4(a[4 * q], a[4 * q + 1], a[4 * q + 2], a[4 * q + 3]);
#pragma unroll
      for (int c = 0; c < CB; ++c) s_lt[c][r] = a[c];   // s_lt[c][r] = L(r, c)
      s_rpv[J + r] = myrp;
      s_csv[J + r] = mycs;
    }
  };
  // X_JJ = L_JJ^-1 by one warp, by columns: lane r holds column r, x[i] = X(i, r), zero for
  // i < r, from the rows of L_JJ in A and the reciprocal pivots.
  auto xjj_block = [&](int J) {
    const int r = lane & 15;
    float x[CB];
#pragma unroll
    for (int i = 0; i < CB; ++i) {
      const float4* li = reinterpret_cast<const float4*>(arow(J + i) + J);
      float lrow[CB];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 t = li[q];
        lrow[4 * q] = t.x; lrow[4 * q + 1] = t.y; lrow[4 * q + 2] = t.z; lrow[4 * q + 3] = t.w;
      }
      float v0 = 0.0f, v1 = 0.0f;
#pragma unroll
      for (int k = 0; k < i; ++k) {
        if (k & 1) v1 = fmaf(lrow[k], x[k], v1);
        else v0 = fmaf(lrow[k], x[k], v0);
      }
      const float rp = s_rpv[J + i];
      x[i] = (i > r) ? -(v0 + v1) * rp : (i == r ? rp : 0.0f);
    }
    if (lane < CB) {
#pragma unroll
      for (int i = 0; i < CB; ++i) xrow(J + i)[J + r] = x[i];
    }
  };
  // A_ik -= L_iJ . L_kJ for rows i0, i0 + 1 and columns k = k0, k0 + kstep, ... <= i
  auto update_rows = [&](int J, int i0, int k0, int kstep) {
    const int i1 = i0 + 1;
    const float4* p0 = reinterpret_cast<const float4*>(arow(i0) + J);
    const float4* p1 = reinterpret_cast<const float4*>(arow(i1) + J);
    const float4 u0 = p0[0], u1 = p0[1], u2 = p0[2], u3 = p0[3];
    const float4 w0 = p1[0], w1 = p1[1], w2 = p1[2], w3 = p1[3];
    for (int k = k0; k <= i1; k += kstep) {
      const float4* pk = reinterpret_cast<const float4*>(arow(k) + J);
      const float4 k0v = pk[0], k1 = pk[1], k2 = pk[2], k3 = pk[3];
      const float a0 = dot4(u0, k0v, dot4(u1, k1, 0.0f)) + dot4(u2, k2, dot4(u3, k3, 0.0f));
      const float a1 = dot4(w0, k0v, dot4(w1, k1, 0.0f)) + dot4(w2, k2, dot4(w3, k3, 0.0f));
      if (k <= i0) arow(i0)[k] -= a0;
      arow(i1)[k] -= a1;
    }
  };

  // Off-diagonal blocks of X = L^-1, block row I (16 rows) from the block rows above it:
  // S(r, c) = sum_{c<=k<I} L(I+r, k) X(k, c) into A's scratch upper triangle
  // (A[c][I + r], c < I; a separate 16-row block in the packed form), then
  // X(I+r, c) = -sum_{t<=r} X_II(r, t) S(t, c).  Run by threads t < nt of the caller.
  // S in 4 x 4 tiles (rows 4 rg .. 4 rg + 3, columns c0 = 4 cg .. c0 + 3), consecutive
  // lanes on consecutive column groups (their rows of X fall in distinct banks); the k
  // range of a tile, [c0, I) (X(k, c) = 0 for k < c), is split into two halves on
  // neighbouring lanes, summed by one shuffle (2 I is a multiple of 32: whole warps).
  auto inverse_s = [&](int I, int t, int nt) {
    const int ncg = I / 4;
    for (int u = t; u < 2 * I; u += nt) {
      const int tile = u >> 1, h = u & 1;
      const int cg = tile % ncg, rg = tile / ncg;
      const int c0 = 4 * cg;
      const int half4 = (((I - c0) >> 2) + 1) >> 1;
      const int kb = h ? c0 + 4 * half4 : c0, ke = h ? I : c0 + 4 * half4;
      const float* l0 = arow(I + 4 * rg);
      const float* l1 = arow(I + 4 * rg + 1);
      const float* l2 = arow(I + 4 * rg + 2);
      const float* l3 = arow(I + 4 * rg + 3);
      float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0, s2 = s0, s3 = s0;   // rows of the tile
      for (int k = kb; k < ke; k += 4) {
        const float4 a0 = *reinterpret_cast<const float4*>(l0 + k);
        const float4 a1 = *reinterpret_cast<const float4*>(l1 + k);
        const float4 a2 = *reinterpret_cast<const float4*>(l2 + k);
        const float4 a3 = *reinterpret_cast<const float4*>(l3 + k);
        const float4 x0 = *reinterpret_cast<const float4*>(xrow(k) + c0);
        const float4 x1 = *reinterpret_cast<const float4*>(xrow(k + 1) + c0);
        const float4 x2 = *reinterpret_cast<const float4*>(xrow(k + 2) + c0);
        const float4 x3 = *reinterpret_cast<const float4*>(xrow(k + 3) + c0);
        s0 = axpy4(a0.x, x0, s0); s1 = axpy4(a1.x, x0, s1); s2 = axpy4(a2.x, x0, s2); s3 = axpy4(a3.x, x0, s3);
        s0 = axpy4(a0.y, x1, s0); s1 = axpy4(a1.y, x1, s1); s2 = axpy4(a2.y, x1, s2); s3 = axpy4(a3.y, x1, s3);
        s0 = axpy4(a0.z, x2, s0); s1 = axpy4(a1.z, x2, s1); s2 = axpy4(a2.z, x2, s2); s3 = axpy4(a3.z, x2, s3);
        s0 = axpy4(a0.w, x3, s0); s1 = axpy4(a1.w, x3, s1); s2 = axpy4(a2.w, x3, s2); s3 = axpy4(a3.w, x3, s3);
      }
      auto pair_sum = [](float4 v) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, 1);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, 1);
        v.z += __shfl_xor_sync(0xffffffffu, v.z, 1);
        v.w += __shfl_xor_sync(0xffffffffu, v.w, 1);
        return v;
      };
      s0 = pair_sum(s0); s1 = pair_sum(s1); s2 = pair_sum(s2); s3 = pair_sum(s3);
      // S(t, c) goes to srow(c)[t]; lane h writes columns c0 + 2 h and c0 + 2 h + 1
      constexpr int SLD = PACKED ? 20 : LD;
      float* d = (PACKED ? Sb + c0 * 20 : A + c0 * LD + I) + 4 * rg;
      if (h == 0) {
        *reinterpret_cast<float4*>(d) = make_float4(s0.x, s1.x, s2.x, s3.x);
        *reinterpret_cast<float4*>(d + SLD) = make_float4(s0.y, s1.y, s2.y, s3.y);
      } else {
        *reinterpret_cast<float4*>(d + 2 * SLD) = make_float4(s0.z, s1.z, s2.z, s3.z);
        *reinterpret_cast<float4*>(d + 3 * SLD) = make_float4(s0.w, s1.w, s2.w, s3.w);
      }
    }
  };
  auto inverse_x = [&](int I, int t, int nt) {
    const int r = t & 15;
    const float4* xr = reinterpret_cast<const float4*>(xrow(I + r) + I);
    const float4 x0 = xr[0], x1 = xr[1], x2 = xr[2], x3 = xr[3];   // X_II row r (zero beyond r)
    for (int c = t >> 4; c < I; c += nt >> 4) {
      const float4* sc = reinterpret_cast<const float4*>(PACKED ? Sb + c * 20 : A + c * LD + I);
      const float v = dot4(x0, sc[0], dot4(x2, sc[2], 0.0f)) + dot4(x1, sc[1], dot4(x3, sc[3], 0.0f));
      xrow(I + r)[c] = -v;
    }
  };

  // Right-looking blocked factorisation with look-ahead: after the panel of block column
  // J and the update of the next diagonal block, warp 0 factors that block while the
  // other warps update the rest of the trailing triangle and form block row J of the
  // inverse.
  if (warp == 0) diag_factor(0);
  __syncthreads();
#pragma unroll 1
  for (int jb = 0; jb + 1 < NB; ++jb) {
    const int J = jb * CB, s0 = J + CB;
    // panel, in place: L_iJ = A_iJ L_JJ^-T by forward substitution, one thread per row
    // (a floored pivot's column is zero)
    for (int i = s0 + tid; i < LP; i += 512) {
      float* ai = arow(i) + J;
      float a[CB], rp[CB];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 t = reinterpret_cast<const float4*>(ai)[q];
        a[4 * q] = t.x; a[4 * q + 1] = t.y; a[4 * q + 2] = t.z; a[4 * q + 3] = t.w;
        const float4 u = reinterpret_cast<const float4*>(s_csv + J)[q];
        rp[4 * q] = u.x; rp[4 * q + 1] = u.y; rp[4 * q + 2] = u.z; rp[4 * q + 3] = u.w;
      }
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        const float lc = a[c] * rp[c];
        a[c] = lc;
        if (c + 1 < CB) {
          float lt[CB];   // column c of L_JJ
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 t = reinterpret_cast<const float4*>(s_lt[c < CB - 1 ? c : 0])[q];
            lt[4 * q] = t.x; lt[4 * q + 1] = t.y; lt[4 * q + 2] = t.z; lt[4 * q + 3] = t.w;
          }
#pragma unroll
          for (int c2 = c + 1; c2 < CB; ++c2) a[c2] = fmaf(-lc, lt[c2], a[c2]);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        reinterpret_cast<float4*>(ai)[q] = make_float4(a[4 * q], a[4 * q + 1], a[4 * q + 2], a[4 * q + 3]);
    }
    __syncthreads();
    // the next diagonal block's lower triangle (136 entries), one per thread
    if (tid < CB * (CB + 1) / 2) {
      int i = (int)((sqrtf(8.0f * tid + 1.0f) - 1.0f) * 0.5f);
      if ((i + 1) * (i + 2) / 2 <= tid) ++i;
      if (i * (i + 1) / 2 > tid) --i;
      const int k = tid - i * (i + 1) / 2;
      const float4* pi = reinterpret_cast<const float4*>(arow(s0 + i) + J);
      const float4* pk = reinterpret_cast<const float4*>(arow(s0 + k) + J);
      const float v = dot4(pi[0], pk[0], dot4(pi[1], pk[1], 0.0f)) + dot4(pi[2], pk[2], dot4(pi[3], pk[3], 0.0f));
      arow(s0 + i)[s0 + k] -= v;
    }
    __syncthreads();
    // The trailing update runs on 11 of the 12 warps that do not share warp 0's scheduler
    // (warp w issues from sub-partition w mod 4), so the latency-bound factorisation of
    // the diagonal block is not slowed by their instructions; the twelfth inverts L_JJ.
    // They then form block row J of X = L^-1: it needs X above it, L's rows J .. J + 15
    // left of J (final since the previous panel) and X_JJ, and nothing that this step
    // writes.
    if (warp == 0) {
      diag_factor(s0);
    } else if (warp & 3) {
      constexpr int NTW = NW - NW / 4;
      const int tw = warp - (warp >> 2) - 1;
      if (!PACKED && tw == 0) {
        xjj_block(J);
      } else {
        // in the packed form L^-1 is formed by trinv_kernel afterwards: all 12 warps update
        const int t0 = PACKED ? tw : tw - 1, ntr = PACKED ? NTW : NTW - 1;
        for (int ip = t0; 2 * ip < LP - s0 - CB; ip += ntr) update_rows(J, s0 + CB + 2 * ip, s0 + lane, 32);
      }
      asm volatile("bar.sync 1, %0;" ::"n"(NTW * 32) : "memory");   // the trailing warps only
      if (!PACKED && jb >= 1) {
        const int tt = tw * 32 + lane;
        inverse_s(J, tt, NTW * 32);
        asm volatile("bar.sync 1, %0;" ::"n"(NTW * 32) : "memory");
        inverse_x(J, tt, NTW * 32);
      }
    }
    __syncthreads();
  }

  // the last diagonal block and block row of the inverse
  if (!PACKED) {
    if (warp == 0) xjj_block(CB * (NB - 1));
    __syncthreads();
    inverse_s(CB * (NB - 1), tid, 512);
    __syncthreads();
    inverse_x(CB * (NB - 1), tid, 512);
    __syncthreads();
  }

  // outputs: R = L^T, R^-1 = X^T restricted to l x l (and racc <- R when racc_init).  A
  // thread reads four consecutive columns a of row b of L and X (lanes on consecutive
  // rows: distinct banks) and writes them to rows a of the outputs (coalesced over b).
  // In the packed form R^-1 comes from trinv_kernel.
  {
    const bool rinit = racc != nullptr && racc_init;
    for (int t = tid; t < LP * (LP / 4); t += 512) {
      const int b = t % LP, a4 = 4 * (t / LP);
      float4 lv = make_float4(0.f, 0.f, 0.f, 0.f), xv = lv;
      if (a4 <= b && b < l) {
        lv = *reinterpret_cast<const float4*>(arow(b) + a4);
        if (!PACKED) xv = *reinterpret_cast<const float4*>(xrow(b) + a4);
      }
      const float lq[4] = {lv.x, lv.y, lv.z, lv.w}, xq[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int a = a4 + q;
        const bool up = (a < l && b < l && b >= a);
        r_out[a * LP + b] = up ? lq[q] : 0.0f;
        if (!PACKED) rinv[a * LP + b] = up ? xq[q] : 0.0f;
        if (rinit) racc[a * LP + b] = up ? lq[q] : 0.0f;
      }
    }
    if (rinit) return;
  }
  if (racc) {
    __syncthreads();
    // stage the old racc (upper, l x l) in the free X space, then racc <- R racc in
    // 1 x 4 strips: P(a, b0..b0+3) = sum_{a<=c<=b0+3} R(a, c) Ro(c, b0..b0+3)
#pragma unroll 1
    for (int r0 = 0; r0 < NB; r0 += RCH) {
      float v[RCH][NCOL];
#pragma unroll
      for (int r = 0; r < RCH; ++r)
#pragma unroll
        for (int c = 0; c < NCOL; ++c) {
          const int i = warp + NW * (r0 + r), j = lane + 32 * c;
          v[r][c] = (i < LP && j < LP) ? racc[i * LP + j] : 0.0f;
        }
#pragma unroll
      for (int r = 0; r < RCH; ++r)
#pragma unroll
        for (int c = 0; c < NCOL; ++c) {
          const int i = warp + NW * (r0 + r), j = lane + 32 * c;
          if (i < LP && j < LP) xrow(i)[j] = v[r][c];   // the old racc, staged where X was
        }
    }
    __syncthreads();
    constexpr int NQ = LP / 4;
    for (int t = tid; t < LP * NQ; t += 512) {
      const int a = t / NQ, b0 = 4 * (t - a * NQ);
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f), acc1 = acc;
      if (a < l && b0 + 3 >= a) {
        const int cend = min(b0 + 3, l - 1);
        int c = a;
        for (; c + 3 <= cend; c += 4) {   // four rows per step, all loads in flight
          const float r0 = arow(c)[a], r1 = arow(c + 1)[a], r2 = arow(c + 2)[a], r3 = arow(c + 3)[a];
          const float4 o0 = *reinterpret_cast<const float4*>(xrow(c) + b0);
          const float4 o1 = *reinterpret_cast<const float4*>(xrow(c + 1) + b0);
          const float4 o2 = *reinterpret_cast<const float4*>(xrow(c + 2) + b0);
          const float4 o3 = *reinterpret_cast<const float4*>(xrow(c + 3) + b0);
          acc = axpy4(r0, o0, acc);
          acc1 = axpy4(r1, o1, acc1);
          acc = axpy4(r2, o2, acc);
          acc1 = axpy4(r3, o3, acc1);
        }
        for (; c <= cend; ++c)
          acc = axpy4(arow(c)[a], *reinterpret_cast<const float4*>(xrow(c) + b0), acc);
        acc.x += acc1.x; acc.y += acc1.y; acc.z += acc1.z; acc.w += acc1.w;
      }
      float4 o;
      o.x = (a < l && b0 < l && b0 >= a) ? acc.x : 0.0f;
      o.y = (a < l && b0 + 1 < l && b0 + 1 >= a) ? acc.y : 0.0f;
      o.z = (a < l && b0 + 2 < l && b0 + 2 >= a) ? acc.z : 0.0f;
      o.w = (a < l && b0 + 3 < l && b0 + 3 >= a) ? acc.w : 0.0f;
      *reinterpret_cast<float4*>(racc + a * LP + b0) = o;
    }
  }
}

// X = L^-1 for the packed form (l_p > 160), from R = L^T (l_p x l_p, upper, zero beyond
// l) after the factorisation: CTA c forms column block c of X (16 columns, rows 16 c ..
// l_p - 1) by block forward substitution, X_cc = L_cc^-1 and
//   X_Ic = -X_II sum_{c<=K<I} L_IK X_Kc,   I = c + 1 .. NB - 1,
// and writes rows 16 c .. 16 c + 15 of R^-1 = X^T.  The diagonal inverses X_II come from
// the rows of L_II by columns (one warp per block), with L treated as the identity beyond
// l.  The column blocks are independent: NB CTAs run them side by side.
template <int NB>
__host__ __device__ constexpr int trinv_ldl() { return CB * (NB - 1) + 4; }
template <int NB>
constexpr size_t trinv_smem() {
  return (size_t)(2 * NB * CB * CB + CB * trinv_ldl<NB>() + CB * CB) * sizeof(float);
}

template <int NB>
__global__ void __launch_bounds__(256, 1) trinv_kernel(const float* __restrict__ r, int l,
                                                    float* __restrict__ rinv) {
  constexpr int LP = CB * NB, LDL = trinv_ldl<NB>();
  extern __shared__ __align__(16) float tsm[];
  const int c = blockIdx.x, nbr = NB - c;
  float* Xs = tsm;                       // X(16 c + i, 16 c + t) at [i][t], i < 16 nbr
  float* Xd = Xs + NB * CB * CB;         // X_II for I = c + ii at [ii][row][col]
  float* Ls = Xd + NB * CB * CB;         // L(16 I + row, 16 c + k) at [row][k]
  float* Ts = Ls + CB * LDL;             // 16 x 16
  pdl_wait();
  pdl_trigger();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rr = lane & 15;
  for (int ii = warp; ii < nbr; ii += 8) {
    const int I = c + ii;
    float lrow[CB];   // row rr of L_II
#pragma unroll
    for (int t = 0; t < CB; ++t) {
      const int gi = CB * I + rr, gj = CB * I + t;
      float v = (t <= rr) ? r[(int64_t)gj * LP + gi] : 0.0f;
      if (gi >= l || gj >= l) v = (gi == gj) ? 1.0f : 0.0f;
      lrow[t] = v;
    }
    // lane rr forms column rr of X_II: x[i] = X(i, rr), zero above the diagonal
    float x[CB];
#pragma unroll
    for (int i = 0; i < CB; ++i) {
      float v0 = 0.0f, v1 = 0.0f;
#pragma unroll
      for (int k = 0; k < i; ++k) {
        const float lik = __shfl_sync(0xffffffffu, lrow[k], i);
        if (k & 1) v1 = fmaf(lik, x[k], v1);
        else v0 = fmaf(lik, x[k], v0);
      }
      const float lii = __shfl_sync(0xffffffffu, lrow[i], i);
      x[i] = (i > rr) ? -(v0 + v1) / lii : (i == rr ? 1.0f / lii : 0.0f);
    }
    if (lane < CB) {
#pragma unroll
      for (int i = 0; i < CB; ++i) Xd[(ii * CB + i) * CB + rr] = x[i];
    }
  }
  __syncthreads();
  Xs[tid] = Xd[tid];   // X_cc (256 threads, 16 x 16)
  __syncthreads();
  for (int ii = 1; ii < nbr; ++ii) {
    const int I = c + ii, kw = CB * ii;
    for (int e = tid; e < kw * CB; e += 256) {   // L_{I, c .. I-1}, read along rows of R
      const int k = e >> 4, q = e & 15;
      Ls[q * LDL + k] = r[(int64_t)(CB * c + k) * LP + CB * I + q];
    }
    __syncthreads();
    {
      const int q = tid >> 4, t = tid & 15;
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
      for (int k = 0; k < kw; k += 4) {
        s0 = fmaf(Ls[q * LDL + k], Xs[k * CB + t], s0);
        s1 = fmaf(Ls[q * LDL + k + 1], Xs[(k + 1) * CB + t], s1);
        s2 = fmaf(Ls[q * LDL + k + 2], Xs[(k + 2) * CB + t], s2);
        s3 = fmaf(Ls[q * LDL + k + 3], Xs[(k + 3) * CB + t], s3);
      }
      Ts[q * CB + t] = (s0 + s1) + (s2 + s3);
    }
    __syncthreads();
    {
      const int q = tid >> 4, t = tid & 15;
      float s = 0.0f;
#pragma unroll
      for (int u = 0; u < CB; ++u) s = fmaf(Xd[(ii * CB + q) * CB + u], Ts[u * CB + t], s);
      Xs[(kw + q) * CB + t] = -s;
    }
    __syncthreads();
  }
  // rows 16 c .. 16 c + 15 of R^-1: R^-1(a, b) = X(b, a) for a <= b < l
  for (int e = tid; e < CB * LP; e += 256) {
    const int t = e / LP, b = e - t * LP, a = CB * c + t;
    float v = 0.0f;
    if (a < l && b < l && b >= a) v = Xs[(b - CB * c) * CB + t];
    rinv[(int64_t)a * LP + b] = v;
  }
}

__global__ void to_bf16_t_kernel(const float* __restrict__ x, int64_t rows, int lp,
                                 __nv_bfloat16* __restrict__ out, int64_t ld_t, int split,
                                 int lo_off) {
  __shared__ float tile[32][33];
  pdl_wait();
  pdl_trigger();
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

__device__ __forceinline__ void split_one(float v, __nv_bfloat16* hi_out, __nv_bfloat16* lo_out) {
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  *hi_out = hi;
  if (lo_out) *lo_out = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// A (float32) -> hi = bf16(A) and, with with_lo, lo = bf16(A - hi) rows * ld_out elements
// further.  One row per block iteration; four columns per thread when every row starts
// on a 16-byte boundary on both sides.
__global__ void split_bf16_kernel(const float* __restrict__ x, int64_t rows, int64_t cols,
                                  int64_t ld, __nv_bfloat16* __restrict__ out, int64_t ld_out,
                                  int with_lo, int vec4, int64_t lo_off) {
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    const float* xr = x + r * ld;
    __nv_bfloat16* hr = out + r * ld_out;
    __nv_bfloat16* lr = hr + lo_off;
    if (vec4) {
      for (int64_t c = 4 * (int64_t)threadIdx.x; c < cols; c += 4 * (int64_t)blockDim.x) {
        const float4 v = *reinterpret_cast<const float4*>(xr + c);
        __align__(8) __nv_bfloat16 h[4], l[4];
        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) split_one(vv[i], &h[i], &l[i]);
        *reinterpret_cast<uint2*>(hr + c) = *reinterpret_cast<const uint2*>(h);
        if (with_lo) *reinterpret_cast<uint2*>(lr + c) = *reinterpret_cast<const uint2*>(l);
      }
    } else {
      for (int64_t c = threadIdx.x; c < cols; c += blockDim.x)
        split_one(xr[c], hr + c, with_lo ? lr + c : nullptr);
    }
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
template <int NB>
size_t chol_smem() {
  return NB > 10 ? (size_t)(pk_off(CB * NB) + 20 * CB * NB) * sizeof(float)
                 : (size_t)2 * (CB * NB) * (CB * NB + 4) * sizeof(float);
}

template <int NB>
cudaError_t prep_chol() {
  cudaError_t e = cudaFuncSetAttribute(cholesky_blocked_kernel<NB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chol_smem<NB>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(trinv_kernel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)trinv_smem<NB>());
}

template <int LP>
cudaError_t prep_tri() {
  cudaError_t e = cudaFuncSetAttribute(orth_tri_kernel<LP, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       TriCfg<LP, true>::SMEM);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(orth_tri_kernel<LP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              TriCfg<LP, false>::SMEM);
}

template <bool APPLY>
cudaError_t launch_tri(const float* y, int splits, int64_t split_stride, float* q, int64_t rows,
                       int lp, const float* rinv, float* gpart, int nblk, int do_gram,
                       cudaStream_t st) {
  const int64_t rpb = round_up(cdiv(rows, nblk), TR_ROWS);
#define RSVD_TRI_CASE(LP)                                                                     \
  case LP:                                                                                   \
    return launch_pdl(orth_tri_kernel<LP, APPLY>, dim3(nblk), dim3(TriCfg<LP, APPLY>::T),    \
                      (size_t)TriCfg<LP, APPLY>::SMEM, st, y, splits, split_stride, q, rows, rinv, \
                      gpart, rpb, do_gram);
  switch (lp) {
    RSVD_TRI_CASE(16) RSVD_TRI_CASE(32) RSVD_TRI_CASE(48) RSVD_TRI_CASE(64)
    RSVD_TRI_CASE(80) RSVD_TRI_CASE(96) RSVD_TRI_CASE(112) RSVD_TRI_CASE(128)
    default: return cudaErrorInvalidValue;
  }
#undef RSVD_TRI_CASE
}

cudaError_t prepare_orth() {
  cudaError_t e;
  if ((e = prep_tri<16>()) != cudaSuccess || (e = prep_tri<32>()) != cudaSuccess ||
      (e = prep_tri<48>()) != cudaSuccess || (e = prep_tri<64>()) != cudaSuccess ||
      (e = prep_tri<80>()) != cudaSuccess || (e = prep_tri<96>()) != cudaSuccess ||
      (e = prep_tri<112>()) != cudaSuccess || (e = prep_tri<128>()) != cudaSuccess)
    return e;
  if ((e = prep_chol<1>()) != cudaSuccess || (e = prep_chol<2>()) != cudaSuccess ||
      (e = prep_chol<3>()) != cudaSuccess || (e = prep_chol<4>()) != cudaSuccess ||
      (e = prep_chol<5>()) != cudaSuccess || (e = prep_chol<6>()) != cudaSuccess ||
      (e = prep_chol<7>()) != cudaSuccess || (e = prep_chol<8>()) != cudaSuccess ||
      (e = prep_chol<9>()) != cudaSuccess || (e = prep_chol<10>()) != cudaSuccess ||
      (e = prep_chol<11>()) != cudaSuccess || (e = prep_chol<12>()) != cudaSuccess ||
      (e = prep_chol<13>()) != cudaSuccess || (e = prep_chol<14>()) != cudaSuccess ||
      (e = prep_chol<15>()) != cudaSuccess || (e = prep_chol<16>()) != cudaSuccess)
    return e;
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

cudaError_t launch_apply_gram(const float* y, float* q, int64_t rows, int lp, const float* rinv,
                              float* gpart, int nblk, int do_gram, cudaStream_t st) {
  return launch_tri<true>(y, 1, 0, q, rows, lp, rinv, gpart, nblk, do_gram, st);
}

cudaError_t launch_gram_tri(const float* src, int splits, int64_t split_stride, float* y_out,
                            int64_t rows, int lp, float* gpart, int nblk, cudaStream_t st) {
  return launch_tri<false>(src, splits, split_stride, y_out, rows, lp, nullptr, gpart, nblk, 1, st);
}

cudaError_t launch_gram_reduce(const float* gpart, int nblk, int lp, float* g, cudaStream_t st) {
  const int64_t n = (int64_t)lp * lp;
  return launch_pdl(gram_reduce_kernel, dim3((unsigned)cdiv(n, 32)), dim3(512), 0, st, gpart, nblk,
                    lp, g);
}

cudaError_t launch_trinv_upper(const float* r, int l, int lp, float* rinv, cudaStream_t st) {
#define RSVD_TRINV_CASE(NB) \
  case NB:                  \
    return launch_pdl(trinv_kernel<NB>, dim3(NB), dim3(256), trinv_smem<NB>(), st, r, l, rinv);
  switch (lp % CB == 0 ? lp / CB : 0) {
    RSVD_TRINV_CASE(1) RSVD_TRINV_CASE(2) RSVD_TRINV_CASE(3) RSVD_TRINV_CASE(4) RSVD_TRINV_CASE(5)
    RSVD_TRINV_CASE(6) RSVD_TRINV_CASE(7) RSVD_TRINV_CASE(8) RSVD_TRINV_CASE(9) RSVD_TRINV_CASE(10)
    RSVD_TRINV_CASE(11) RSVD_TRINV_CASE(12) RSVD_TRINV_CASE(13) RSVD_TRINV_CASE(14)
    RSVD_TRINV_CASE(15) RSVD_TRINV_CASE(16)
    default: return cudaErrorInvalidValue;
  }
#undef RSVD_TRINV_CASE
}

cudaError_t launch_cholesky(const float* g, int l, int lp, int shifted, float* lbuf, float* r_out,
                            float* rinv, float* racc, int racc_init, uint32_t* status,
                            cudaStream_t st) {
  if (lp <= 256 && lp % CB == 0 && lbuf) {
#define RSVD_CHOL_CASE(NB)                                                                  \
  case NB: {                                                                               \
    cudaError_t e = launch_pdl(cholesky_blocked_kernel<NB>, dim3(1), dim3(512), chol_smem<NB>(), st, \
                               g, l, shifted, r_out, rinv, racc, racc_init, status, lbuf);  \
    if (e != cudaSuccess || NB <= 10) return e;                                            \
    return launch_pdl(trinv_kernel<NB>, dim3(NB), dim3(256), trinv_smem<NB>(), st,          \
                      (const float*)r_out, l, rinv);                                       \
  }
    switch (lp / CB) {
      RSVD_CHOL_CASE(1) RSVD_CHOL_CASE(2) RSVD_CHOL_CASE(3) RSVD_CHOL_CASE(4) RSVD_CHOL_CASE(5)
      RSVD_CHOL_CASE(6) RSVD_CHOL_CASE(7) RSVD_CHOL_CASE(8) RSVD_CHOL_CASE(9) RSVD_CHOL_CASE(10)
      RSVD_CHOL_CASE(11) RSVD_CHOL_CASE(12) RSVD_CHOL_CASE(13) RSVD_CHOL_CASE(14)
      RSVD_CHOL_CASE(15) RSVD_CHOL_CASE(16)
      default: break;
    }
#undef RSVD_CHOL_CASE
  }
  const size_t smem = ((size_t)l * (l + 1) / 2 + l + 4 + kMaxL) * sizeof(float);
  cholesky_kernel<<<1, 1024, smem, st>>>(g, l, lp, shifted, lbuf, r_out, rinv, racc, racc_init,
                                         status);
  return cudaGetLastError();
}

cudaError_t launch_to_bf16_t(const float* x, int64_t rows, int lp, __nv_bfloat16* out, int64_t ld_t,
                             int split, int lo_off, cudaStream_t st) {
  const dim3 grid((unsigned)cdiv(rows, 32), (unsigned)cdiv(lp, 32));
  return launch_pdl(to_bf16_t_kernel, grid, dim3(32, 8), 0, st, x, rows, lp, out, ld_t, split, lo_off);
}

cudaError_t launch_split_bf16(const float* x, int64_t rows, int64_t cols, int64_t ld,
                              __nv_bfloat16* out, int64_t ld_out, int with_lo, cudaStream_t st,
                              int64_t lo_off) {
  if (rows * cols == 0) return cudaSuccess;
  if (lo_off < 0) lo_off = rows * ld_out;
  const int vec4 = (cols % 4 == 0 && ld % 4 == 0 && ld_out % 4 == 0 && lo_off % 4 == 0 &&
                    (reinterpret_cast<uintptr_t>(x) & 15) == 0 &&
                    (reinterpret_cast<uintptr_t>(out) & 7) == 0) ? 1 : 0;
  const unsigned grid = (unsigned)(rows < 16 * kNumSMs ? rows : 16 * kNumSMs);
  split_bf16_kernel<<<grid, 256, 0, st>>>(x, rows, cols, ld, out, ld_out, with_lo, vec4, lo_off);
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
