// One-sided Jacobi SVD of the small l x l matrix of Stage B (Algorithm 5.1
// step 2, taken as in Section 3.3.3) on a thread-block cluster, for l <= 256.
//
// Block-parallel ordering: the (padded) columns form 2C blocks of bw columns; the
// C CTAs of the cluster each hold two blocks of X and of the accumulated rotations
// J in shared memory.  A sweep is 2C - 1 rounds of the round-robin tournament over
// the blocks (position 0 fixed, the others moving one place per round): in a round
// each CTA rotates every pair (i, j) with i in its first block and j in its second
// (bw sub-rounds of bw disjoint pairs, one half-warp per pair), then pulls the two
// blocks its positions take next from their holders' shared memory (distributed
// shared memory, double-buffered, one cluster barrier per round).  The pairs inside
// a block are rotated at the start of each sweep.  So every pair of columns meets
// once per sweep, as in the cyclic sweep of the one-CTA kernel, while 2C pairs'
// worth of rotation work runs on C SMs at once and no column is read remotely
// during the rotations.  The rotation is the tan(angle/2) form; a pair counts as
// orthogonal while |x_p . x_q| <= tol ||x_p|| ||x_q||; sweeps end when none rotates.
// Epilogue: sigma_c = ||x_c||, U = X diag(1/sigma), W = J, in descending sigma order; a
// second kernel polishes W by one Newton-Schulz step W <- W (3 I - W^T W) / 2.
#include <cooperative_groups.h>
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace rsvd {
namespace {

constexpr int kMaxLC = 256;
constexpr int kSweepsC = 40;
constexpr int kThreadsC = 256;   // 16 half-warps: one per pair of a sub-round (bw <= 16)
constexpr int kMaxCluster = 8;

template <int VPL>
__device__ __forceinline__ void ldcol(const float* p, int hl, float (&u)[4 * VPL]) {
#pragma unroll
  for (int k = 0; k < VPL; ++k) {
    const float4 a = reinterpret_cast<const float4*>(p)[hl + 16 * k];
    u[4 * k] = a.x; u[4 * k + 1] = a.y; u[4 * k + 2] = a.z; u[4 * k + 3] = a.w;
  }
}

template <int VPL>
__device__ __forceinline__ void stcol(float* p, int hl, const float (&u)[4 * VPL]) {
#pragma unroll
  for (int k = 0; k < VPL; ++k)
    reinterpret_cast<float4*>(p)[hl + 16 * k] =
        make_float4(u[4 * k], u[4 * k + 1], u[4 * k + 2], u[4 * k + 3]);
}

// [u v] <- [u v] [[c, s], [-s, c]] in the tan(theta / 2) form, tau = s / (1 + c):
// u - s (tau u + v), v + s (u - tau v).  Its scaling error is (c^2 + s^2 - 1) times
// (1 - c) / (1 + c), about theta^2 / 4 of that of the plain form, which keeps column norms
// from drifting over the many small rotations of the last sweeps.
template <int VPL>
__device__ __forceinline__ void rotcols(float (&u)[4 * VPL], float (&v)[4 * VPL], float sn, float tau) {
#pragma unroll
  for (int i = 0; i < 4 * VPL; ++i) {
    const float uu = u[i], vv = v[i];
    u[i] = uu - sn * fmaf(tau, uu, vv);
    v[i] = vv + sn * fmaf(-tau, vv, uu);
  }
}

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// The rotation (s, tau = s / (1 + c)) that makes two columns with squared norms a, b and
// inner product g orthogonal; false when they already count as orthogonal,
// g^2 <= tol^2 a b.
// a, b, g are first scaled by the power of two that puts max(a, b) in [1, 2) (exact), so
// neither the test nor the angle underflows for tiny columns.  t = tan(theta) is the
// root of t^2 + 2 zeta t - 1 = 0, zeta = (b - a) / (2 g), with |theta| <= pi/4, taken as
// t = sign(b - a) 2 g / (|b - a| + sqrt((b - a)^2 + 4 g^2)) from approximate reciprocals
// and square roots: any angle gives an orthogonal transform, only how far the pair's new
// inner product is from zero depends on its accuracy.  c = 1 / sqrt(1 + t^2) gets one
// Newton step, so that c^2 + s^2 = 1 to rounding and column norms do not drift.
__device__ __forceinline__ bool jacobi_angle(float a, float b, float g, float tol2, float& sn,
                                             float& tau) {
  const int e = min((__float_as_int(fmaxf(a, b)) >> 23) & 0xff, 253);
  const float f = __int_as_float((254 - e) << 23);
  a *= f;
  b *= f;
  g *= f;
  if (!(g * g > (tol2 * a) * b)) return false;   // also false for g = 0 and NaN
  const float d = b - a;
  const float h = fmaf(d, d, 4.0f * g * g);
  const float r = h * rsqrtf(h);
  float t = 2.0f * g * rcp_approx(fabsf(d) + r);
  t = d < 0.0f ? -t : t;
  const float w = fmaf(t, t, 1.0f);
  float cc = rsqrtf(w);
  cc = cc * fmaf(-0.5f * w, cc * cc, 1.5f);
  sn = cc * t;
  tau = sn * rcp_approx(1.0f + cc);
  return true;
}

// Squared norms and inner product of two columns held by a half-warp, summed over it.
template <int VPL>
__device__ __forceinline__ void col_dots(const float (&u)[4 * VPL], const float (&v)[4 * VPL],
                                         unsigned hmask, float& a, float& b, float& g) {
  float a0 = 0.f, b0 = 0.f, g0 = 0.f, a1 = 0.f, b1 = 0.f, g1 = 0.f;
#pragma unroll
  for (int i = 0; i < 4 * VPL; i += 2) {
    a0 = fmaf(u[i], u[i], a0);
    b0 = fmaf(v[i], v[i], b0);
    g0 = fmaf(u[i], v[i], g0);
    a1 = fmaf(u[i + 1], u[i + 1], a1);
    b1 = fmaf(v[i + 1], v[i + 1], b1);
    g1 = fmaf(u[i + 1], v[i + 1], g1);
  }
  a = a0 + a1;
  b = b0 + b1;
  g = g0 + g1;
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    a += __shfl_xor_sync(hmask, a, o);
    b += __shfl_xor_sync(hmask, b, o);
    g += __shfl_xor_sync(hmask, g, o);
  }
}

// Rotate columns xp, xq (and jp, jq) of shared memory so that they become orthogonal,
// by one half-warp (hl = lane within it, hmask = its lanes).  True when rotated.
template <int VPL>
__device__ __forceinline__ bool pair_rotate(float* xp, float* xq, float* jp, float* jq, int hl,
                                            unsigned hmask, float tol2) {
  float u[4 * VPL], v[4 * VPL], ju[4 * VPL], jv[4 * VPL];
  ldcol<VPL>(xp, hl, u);
  ldcol<VPL>(xq, hl, v);
  ldcol<VPL>(jp, hl, ju);
  ldcol<VPL>(jq, hl, jv);
  float a, b, g, sn, tau;
  col_dots<VPL>(u, v, hmask, a, b, g);
  if (!jacobi_angle(a, b, g, tol2, sn, tau)) return false;
  rotcols<VPL>(u, v, sn, tau);
  rotcols<VPL>(ju, jv, sn, tau);
  stcol<VPL>(xp, hl, u);
  stcol<VPL>(xq, hl, v);
  stcol<VPL>(jp, hl, ju);
  stcol<VPL>(jq, hl, jv);
  return true;
}

// Position p of the tournament is held by CTA p (slot 0) for p < C, else by CTA
// 2C - 1 - p (slot 1).  Moving one place: position 1 takes the block of position
// 2C - 1, position p >= 2 that of p - 1, position 0 keeps its block.
__device__ __forceinline__ int src_position(int p, int nblk) {
  return p == 0 ? 0 : (p == 1 ? nblk - 1 : p - 1);
}

// One matrix per cluster: the grid's first cluster takes job0, a second one job1 (two
// independent SVDs of the same size in one launch).
struct JacobiJob {
  const float* x;
  float* ut;
  float* s;
  float* w;
};

template <int VPL>
__global__ void __launch_bounds__(kThreadsC) jacobi_block_kernel(
    JacobiJob job0, JacobiJob job1, int64_t ldx, int transposed, int l, int lp, int bw,
    uint32_t* status, uint32_t* info, float tol2) {
  constexpr int LR = 64 * VPL;   // rows per stored column (zero beyond l)
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const JacobiJob& job = (int)blockIdx.x < C ? job0 : job1;
  const float* __restrict__ x = job.x;
  float* __restrict__ ut = job.ut;
  float* __restrict__ s = job.s;
  float* __restrict__ w = job.w;
  const int nblk = 2 * C;
  const int slot_floats = 2 * bw * LR;   // X block then J block
  extern __shared__ __align__(16) float sm[];
  // buffer b (0/1, double-buffered) slot sl (0/1): X block then J block
  auto buf = [&](int b, int sl) { return sm + (2 * b + sl) * slot_floats; };
  __shared__ int s_rot[2];
  __shared__ int s_any;
  __shared__ float s_sig[32];
  __shared__ float s_sig_all[kMaxLC];
  const int tid = threadIdx.x;
  const int hw = tid >> 4, hl = tid & 15;
  const int lane = tid & 31, warp = tid >> 5;
  const unsigned hmask = 0xFFFFu << (lane & 16);

  // load: slot 0 holds block `rank`, slot 1 block nblk - 1 - rank
  for (int sl = 0; sl < 2; ++sl) {
    const int blk = sl == 0 ? rank : nblk - 1 - rank;
    float* X = buf(0, sl);
    float* Jm = X + bw * LR;
    for (int e = tid; e < bw * LR; e += kThreadsC) {
      const int i = e / LR, r = e - i * LR;
      const int c = blk * bw + i;
      float v = 0.0f;
      if (c < l && r < l) v = transposed ? x[(int64_t)c * ldx + r] : x[(int64_t)r * ldx + c];
      X[e] = v;
      Jm[e] = (c < l && r == c) ? 1.0f : 0.0f;
    }
  }
  if (tid < 2) s_rot[tid] = 0;
  int cur = 0;
  cluster.sync();

  const int be = bw + (bw & 1);
  int sweep = 0;
  for (; sweep < kSweepsC; ++sweep) {
    const int par = sweep & 1;
    bool rotated = false;
    // pairs inside each block: round-robin over be positions, both slots at once
    for (int rr = 0; rr < be - 1; ++rr) {
      const int half = be >> 1;
      if (hw < 2 * half) {
        const int sl = hw / half, k = hw - sl * half;
        const int p = (k == 0) ? 0 : ((k - 1 + rr) % (be - 1)) + 1;
        const int kq = be - 1 - k;
        const int q = (kq == 0) ? 0 : ((kq - 1 + rr) % (be - 1)) + 1;
        if (p < bw && q < bw) {
          float* X = buf(cur, sl);
          float* Jm = X + bw * LR;
          rotated |= pair_rotate<VPL>(X + p * LR, X + q * LR, Jm + p * LR, Jm + q * LR, hl, hmask, tol2);
        }
      }
      __syncthreads();
    }
    for (int round = 0; round < nblk - 1; ++round) {
      // Half-warp h keeps column h of the first block (X and J) in registers for the
      // round and meets column (h + sub) mod bw of the second block in sub-round sub;
      // that column comes from half-warp h + 1 of the previous sub-round.
      float* X0 = buf(cur, 0);
      float* X1 = buf(cur, 1);
      float* J0 = X0 + bw * LR;
      float* J1 = X1 + bw * LR;
      const bool act = hw < bw;
      float xr[4 * VPL], jr[4 * VPL];
      if (act) {
        ldcol<VPL>(X0 + hw * LR, hl, xr);
        ldcol<VPL>(J0 + hw * LR, hl, jr);
      }
      for (int sub = 0; sub < bw; ++sub) {
        if (act) {
          const int q = hw + sub < bw ? hw + sub : hw + sub - bw;
          float v[4 * VPL], jv[4 * VPL];
          ldcol<VPL>(X1 + q * LR, hl, v);
          ldcol<VPL>(J1 + q * LR, hl, jv);
          float a, b, g, sn, tau;
          col_dots<VPL>(xr, v, hmask, a, b, g);
          if (jacobi_angle(a, b, g, tol2, sn, tau)) {
            rotated = true;
            rotcols<VPL>(xr, v, sn, tau);
            rotcols<VPL>(jr, jv, sn, tau);
            stcol<VPL>(X1 + q * LR, hl, v);
            stcol<VPL>(J1 + q * LR, hl, jv);
          }
        }
        __syncthreads();
      }
      if (act) {
        stcol<VPL>(X0 + hw * LR, hl, xr);
        stcol<VPL>(J0 + hw * LR, hl, jr);
      }
      if (rotated && hl == 0) s_rot[par] = 1;
      cluster.sync();   // every CTA has finished this round: its blocks may be read
      // pull the blocks of the next round into the other buffer
      const int nxt = cur ^ 1;
      for (int sl = 0; sl < 2; ++sl) {
        const int pos = sl == 0 ? rank : nblk - 1 - rank;
        const int sp = src_position(pos, nblk);
        const int src_cta = sp < C ? sp : nblk - 1 - sp;
        const int src_sl = sp < C ? 0 : 1;
        const float4* src = reinterpret_cast<const float4*>(
            cluster.map_shared_rank(buf(cur, src_sl), src_cta));
        float4* dst = reinterpret_cast<float4*>(buf(nxt, sl));
        const int n4 = slot_floats / 4;
        int e = tid;
        for (; e + 3 * kThreadsC < n4; e += 4 * kThreadsC) {
          const float4 a0 = src[e], a1 = src[e + kThreadsC];
          const float4 a2 = src[e + 2 * kThreadsC], a3 = src[e + 3 * kThreadsC];
          dst[e] = a0; dst[e + kThreadsC] = a1; dst[e + 2 * kThreadsC] = a2; dst[e + 3 * kThreadsC] = a3;
        }
        for (; e < n4; e += kThreadsC) dst[e] = src[e];
      }
      cur = nxt;
      // The pulled columns are complete in this CTA before any half-warp rotates them.  No
      // second cluster barrier: a CTA writes its other buffer again only in the next
      // round's pull, after the next cluster barrier, which every CTA reaches only once it
      // has finished this round's pull.
      __syncthreads();
    }
    // after 2C - 1 moves every block is back in its first place; did any CTA rotate?
    if (tid == 0) {
      int any = 0;
      for (int r = 0; r < C; ++r) any |= cluster.map_shared_rank(s_rot, r)[par];
      s_any = any;
      s_rot[par ^ 1] = 0;
    }
    __syncthreads();
    const int any = s_any;
    if (!any) break;
  }
  if (rank == 0 && tid == 0) {
    if (sweep == kSweepsC) set_status(status, ST_JACOBI_NOCONV);
    if (info) atomicMax(info, (uint32_t)(sweep + 1));
  }

  // sigma of the local columns (warp per column), gathered by every CTA
  for (int i = warp; i < 2 * bw; i += kThreadsC / 32) {
    const int sl = i / bw, ci = i - sl * bw;
    const float* col = buf(cur, sl) + ci * LR;
    float a = 0.f;
    for (int e = lane; e < LR; e += 32) a = fmaf(col[e], col[e], a);
    a = warp_sum(a);
    if (lane == 0) s_sig[i] = sqrtf(a);
  }
  cluster.sync();
  for (int c = tid; c < nblk * bw; c += kThreadsC) {
    const int b = c / bw, ci = c - b * bw;
    const int owner = b < C ? b : nblk - 1 - b;
    const int sl = b < C ? 0 : 1;
    s_sig_all[c] = c < l ? cluster.map_shared_rank(s_sig, owner)[sl * bw + ci] : -1.0f;
  }
  cluster.sync();   // no CTA leaves while others read its s_sig
  if (rank == 0)
    for (int e = tid; e < lp * lp; e += kThreadsC) {
      const int r = e / lp, c = e % lp;
      if (r >= l || c >= l) { ut[e] = 0.0f; w[e] = 0.0f; }
    }
  __syncthreads();
  for (int i = warp; i < 2 * bw; i += kThreadsC / 32) {
    const int sl = i / bw, ci = i - sl * bw;
    const int b = sl == 0 ? rank : nblk - 1 - rank;
    const int c = b * bw + ci;
    if (c >= l) continue;
    const float sc = s_sig_all[c];
    int rk = 0;
    for (int c2 = lane; c2 < l; c2 += 32) {
      const float s2 = s_sig_all[c2];
      rk += (s2 > sc || (s2 == sc && c2 < c)) ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rk += __shfl_xor_sync(0xffffffffu, rk, o);
    const float inv = sc > 0.0f ? 1.0f / sc : 0.0f;
    const float* col = buf(cur, sl) + ci * LR;
    const float* jc = buf(cur, sl) + bw * LR + ci * LR;
    for (int e = lane; e < l; e += 32) {
      ut[(int64_t)e * lp + rk] = col[e] * inv;
      w[(int64_t)e * lp + rk] = jc[e];
    }
    if (lane == 0) s[rk] = sc;
  }
}

// W <- W (3 I - W^T W) / 2 on the leading l x l of W (ld lp), a CTA per 16 output
// columns t: G_t = W^T W_t (l x 16; thread c computes row c, reading column c of W
// coalesced across the CTA), then W_t <- 1.5 W_t - 0.5 W G_t (thread r computes
// row r, reading row r of W as float4).  W stays in L2 (<= 256 KB); wout != win.
__global__ void __launch_bounds__(256) ns_polish_kernel(const float* __restrict__ win0, float* __restrict__ wout0,
                                                        const float* __restrict__ win1, float* __restrict__ wout1,
                                                        int l, int lp) {
  // blockIdx.y picks the matrix
  const float* __restrict__ win = blockIdx.y ? win1 : win0;
  float* __restrict__ wout = blockIdx.y ? wout1 : wout0;
  extern __shared__ __align__(16) float psm[];
  float* Wt = psm;              // [l][16]
  float* Gt = psm + 16 * l;     // [l][16]
  const int j0 = blockIdx.x * 16;
  const int tid = threadIdx.x;
  for (int e = tid; e < l * 16; e += 256) {
    const int r = e >> 4, jj = e & 15;
    Wt[e] = (j0 + jj < l) ? win[(int64_t)r * lp + j0 + jj] : 0.0f;
  }
  __syncthreads();
  float acc[16];
  if (tid < l) {
    const int c = tid;
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0f;
    int r = 0;
    for (; r + 16 <= l; r += 16) {
      float wv[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) wv[u] = win[(int64_t)(r + u) * lp + c];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const float4* wt = reinterpret_cast<const float4*>(Wt + (r + u) * 16);
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
          const float4 t = wt[q4];
          acc[4 * q4] = fmaf(wv[u], t.x, acc[4 * q4]);
          acc[4 * q4 + 1] = fmaf(wv[u], t.y, acc[4 * q4 + 1]);
          acc[4 * q4 + 2] = fmaf(wv[u], t.z, acc[4 * q4 + 2]);
          acc[4 * q4 + 3] = fmaf(wv[u], t.w, acc[4 * q4 + 3]);
        }
      }
    }
    for (; r < l; ++r) {
      const float wv = win[(int64_t)r * lp + c];
#pragma unroll
      for (int q = 0; q < 16; ++q) acc[q] = fmaf(wv, Wt[r * 16 + q], acc[q]);
    }
    float4* gt = reinterpret_cast<float4*>(Gt + c * 16);
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4)
      gt[q4] = make_float4(acc[4 * q4], acc[4 * q4 + 1], acc[4 * q4 + 2], acc[4 * q4 + 3]);
  }
  __syncthreads();
  if (tid < l) {
    const int r = tid;
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0f;
    const float* wr = win + (int64_t)r * lp;
    int c = 0;
    for (; c + 16 <= l; c += 16) {   // lp is a multiple of 16: 16-byte aligned rows
      float4 wv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) wv[u] = reinterpret_cast<const float4*>(wr + c)[u];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const float wcu = (u & 3) == 0 ? wv[u >> 2].x : (u & 3) == 1 ? wv[u >> 2].y
                        : (u & 3) == 2 ? wv[u >> 2].z : wv[u >> 2].w;
        const float4* gt = reinterpret_cast<const float4*>(Gt + (c + u) * 16);
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
          const float4 t = gt[q4];
          acc[4 * q4] = fmaf(wcu, t.x, acc[4 * q4]);
          acc[4 * q4 + 1] = fmaf(wcu, t.y, acc[4 * q4 + 1]);
          acc[4 * q4 + 2] = fmaf(wcu, t.z, acc[4 * q4 + 2]);
          acc[4 * q4 + 3] = fmaf(wcu, t.w, acc[4 * q4 + 3]);
        }
      }
    }
    for (; c < l; ++c) {
      const float wcu = wr[c];
#pragma unroll
      for (int q = 0; q < 16; ++q) acc[q] = fmaf(wcu, Gt[c * 16 + q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 16; ++q)
      if (j0 + q < l) wout[(int64_t)r * lp + j0 + q] = 1.5f * Wt[r * 16 + q] - 0.5f * acc[q];
  }
}

template <int VPL>
size_t block_smem(int bw) { return (size_t)4 * 2 * bw * 64 * VPL * sizeof(float); }

template <int VPL>
cudaError_t launch_vpl(int C, int njobs, JacobiJob j0, JacobiJob j1, int64_t ldx, int transposed, int l,
                       int lp, int bw, uint32_t* status, uint32_t* info, float tol2, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C * njobs);
  cfg.blockDim = dim3(kThreadsC);
  cfg.dynamicSmemBytes = block_smem<VPL>(bw);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, jacobi_block_kernel<VPL>, j0, j1, ldx, transposed, l, lp, bw, status,
                            info, tol2);
}

}  // namespace

cudaError_t prepare_jacobi_cluster() {
  cudaError_t e;
  for (const void* fn : {(const void*)jacobi_block_kernel<1>, (const void*)jacobi_block_kernel<2>,
                         (const void*)jacobi_block_kernel<3>, (const void*)jacobi_block_kernel<4>})
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess)
      return e;
  if ((e = cudaFuncSetAttribute(jacobi_block_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)block_smem<1>(16))) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(jacobi_block_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)block_smem<2>(16))) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(jacobi_block_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)block_smem<3>(16))) != cudaSuccess) return e;
  return cudaFuncSetAttribute(jacobi_block_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)block_smem<4>(16));
}

// scratch: lp x lp floats (the unpolished W).  With a second matrix (x_b non-null: the same
// l, lp, ldx and orientation, its own outputs and scratch), both run in one launch, one
// cluster each.
cudaError_t launch_jacobi_cluster(const float* x, int64_t ldx, int transposed, int l, int lp,
                                  float* ut, float* s, float* w, float* scratch, uint32_t* status,
                                  uint32_t* info, cudaStream_t st, const float* x_b, float* ut_b,
                                  float* s_b, float* w_b, float* scratch_b) {
  if (l < 1 || l > kMaxLC || !scratch) return cudaErrorInvalidValue;
  const int njobs = x_b ? 2 : 1;
  if (x_b && !(ut_b && s_b && w_b && scratch_b)) return cudaErrorInvalidValue;
#ifndef RSVD_JACOBI_CSMALL
#define RSVD_JACOBI_CSMALL 4
#endif
  const int C = l <= 128 ? RSVD_JACOBI_CSMALL : kMaxCluster;
  const int bw = (l + 2 * C - 1) / (2 * C);   // <= 16
  const float tol = 8.0f * sqrtf((float)l) * kEpsF32;
  const float tol2 = tol * tol;
  const int vpl = (l + 63) / 64;
  const JacobiJob j0{x, ut, s, scratch};
  const JacobiJob j1 = x_b ? JacobiJob{x_b, ut_b, s_b, scratch_b} : j0;
  cudaError_t e;
  switch (vpl) {
    case 1: e = launch_vpl<1>(C, njobs, j0, j1, ldx, transposed, l, lp, bw, status, info, tol2, st); break;
    case 2: e = launch_vpl<2>(C, njobs, j0, j1, ldx, transposed, l, lp, bw, status, info, tol2, st); break;
    case 3: e = launch_vpl<3>(C, njobs, j0, j1, ldx, transposed, l, lp, bw, status, info, tol2, st); break;
    default: e = launch_vpl<4>(C, njobs, j0, j1, ldx, transposed, l, lp, bw, status, info, tol2, st); break;
  }
  if (e != cudaSuccess) return e;
  // padding of W (rows/columns >= l) is zero in scratch; copy it, then polish the l x l part
  e = cudaMemcpyAsync(w, scratch, sizeof(float) * lp * lp, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && x_b)
    e = cudaMemcpyAsync(w_b, scratch_b, sizeof(float) * lp * lp, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  ns_polish_kernel<<<dim3((l + 15) / 16, njobs), 256, (size_t)32 * l * sizeof(float), st>>>(
      scratch, w, x_b ? scratch_b : scratch, x_b ? w_b : w, l, lp);
  return cudaGetLastError();
}

}  // namespace rsvd
