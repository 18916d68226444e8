// SVD of the small l x l matrix of Stage B (Algorithm 5.1 step 2), taken as
// in Section 3.3.3: B^T = Q_B R_B, then R_B^T = Ut diag(s) W^T, so that
// B = Ut diag(s) (Q_B W)^T.
//
// One-sided (Hestenes) Jacobi in one CTA: the columns of X live in shared
// memory; each sweep visits every column pair once in the round-robin
// ("circle") order, l/2 disjoint pairs per round, one half-warp per pair.  A pair
// (p, q) is rotated when |x_p . x_q| > tol ||x_p|| ||x_q||, with the angle
// from zeta = (||x_q||^2 - ||x_p||^2) / (2 x_p . x_q), t = sign(zeta) /
// (|zeta| + sqrt(1 + zeta^2)).  The same rotations accumulate in J, so that
// X J = U diag(s) and X = U diag(s) J^T.  Sweeps stop when no pair rotates.
// The accumulated J drifts from orthogonality by rounding (about 1e-5 after
// the ~10 l rotations each column receives at l ~ 100); one Newton-Schulz
// step W = J (3 I - J^T J) / 2 at the end brings it back to float32 level.
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {
namespace {

constexpr int kMaxJacobiL = 160;  // X and J both fit in 227 KB of shared memory
constexpr int kMaxSweeps = 40;

__device__ __forceinline__ int rr_player(int pos, int round, int n) {
  return pos == 0 ? 0 : ((pos - 1 + round) % (n - 1)) + 1;
}

__global__ void __launch_bounds__(1024) jacobi_kernel(const float* __restrict__ x, int64_t ldx,
                                                      int transposed, int l, int lp,
                                                      float* __restrict__ ut, float* __restrict__ s,
                                                      float* __restrict__ w, uint32_t* status,
                                                      uint32_t* info, float tol) {
  extern __shared__ __align__(16) float sm[];
  const int le = l + (l & 1);
  float* Xc = sm;                   // [l][l]: Xc[c][e] = X(e, c)
  float* Jc = sm + l * l;           // [l][l]
  float* sig = Jc + l * l;          // [le]
  __shared__ int s_rot;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;

  for (int e = tid; e < l * l; e += nt) {
    const int c = e / l, r = e % l;
    Xc[e] = transposed ? x[(int64_t)c * ldx + r] : x[(int64_t)r * ldx + c];
    Jc[e] = (c == r) ? 1.0f : 0.0f;
  }
  __syncthreads();

  // one half-warp (16 lanes) per column pair: 64 pairs in flight per round
  const int hw = tid >> 4, hl = tid & 15, nhw = nt >> 4;
  const unsigned hmask = 0xFFFFu << (lane & 16);
  int sweep = 0;
  for (; sweep < kMaxSweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < le - 1; ++round) {
      for (int slot = hw; slot < le / 2; slot += nhw) {
        const int p = rr_player(slot, round, le);
        const int q = rr_player(le - 1 - slot, round, le);
        if (p >= l || q >= l) continue;           // the whole half-warp skips together
        float* xp = Xc + p * l;
        float* xq = Xc + q * l;
        float a = 0.f, b = 0.f, g = 0.f;
        for (int e = hl; e < l; e += 16) {
          const float u = xp[e], v = xq[e];
          a = fmaf(u, u, a);
          b = fmaf(v, v, b);
          g = fmaf(u, v, g);
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          a += __shfl_xor_sync(hmask, a, o);
          b += __shfl_xor_sync(hmask, b, o);
          g += __shfl_xor_sync(hmask, g, o);
        }
        if (g == 0.0f || !(fabsf(g) > tol * sqrtf(a * b))) continue;
        // the angle only needs to be close (any angle gives an orthogonal update):
        // fast divisions; cos and tan(angle/2) must be accurate so that the update stays
        // orthogonal (rsqrt refined by one Newton step, an IEEE division for tau)
        const float zeta = __fdividef(b - a, 2.0f * g);
        const float az = fabsf(zeta);
        float t = (az > 1e18f) ? __fdividef(0.5f, az) : __fdividef(1.0f, az + sqrtf(fmaf(az, az, 1.0f)));
        t = copysignf(t, zeta);
        if (zeta == 0.0f) t = 1.0f;
        const float w2 = fmaf(t, t, 1.0f);
        float c = rsqrtf(w2);
        c = c * fmaf(-0.5f * w2, c * c, 1.5f);
        const float sn = c * t;
        const float tau = sn / (1.0f + c);
        if (hl == 0) s_rot = 1;
        float* jp = Jc + p * l;
        float* jq = Jc + q * l;
        for (int e = hl; e < l; e += 16) {
          const float u = xp[e], v = xq[e];
          xp[e] = u - sn * fmaf(tau, u, v);
          xq[e] = v + sn * fmaf(-tau, v, u);
          const float uj = jp[e], vj = jq[e];
          jp[e] = uj - sn * fmaf(tau, uj, vj);
          jq[e] = vj + sn * fmaf(-tau, vj, uj);
        }
      }
      __syncthreads();
    }
    const int rot = s_rot;
    __syncthreads();
    if (!rot) break;
  }
  if (tid == 0) {
    if (sweep == kMaxSweeps) set_status(status, ST_JACOBI_NOCONV);
    if (info) atomicMax(info, (uint32_t)(sweep + 1));
  }

  // singular values = column norms
  for (int c = warp; c < l; c += nw) {
    float a = 0.f;
    for (int e = lane; e < l; e += 32) a = fmaf(Xc[c * l + e], Xc[c * l + e], a);
    a = warp_sum(a);
    if (lane == 0) sig[c] = sqrtf(a);
  }
  __syncthreads();
  // zero the padded frame, then scatter each column to its descending rank
  for (int e = tid; e < lp * lp; e += nt) {
    const int r = e / lp, c = e % lp;
    if (r >= l || c >= l) { ut[e] = 0.0f; w[e] = 0.0f; }
  }
  int* rank_of = reinterpret_cast<int*>(sig + le);  // [l]
  for (int c = warp; c < l; c += nw) {
    const float sc = sig[c];
    int rank = 0;
    for (int c2 = lane; c2 < l; c2 += 32) {
      const float s2 = sig[c2];
      rank += (s2 > sc || (s2 == sc && c2 < c)) ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
    const float inv = sc > 0.0f ? 1.0f / sc : 0.0f;
    for (int e = lane; e < l; e += 32) ut[(int64_t)e * lp + rank] = Xc[c * l + e] * inv;
    if (lane == 0) {
      s[rank] = sc;
      rank_of[c] = rank;
    }
  }
  __syncthreads();
  // Newton-Schulz: G = J^T J (into X's space), W = J (3 I - G) / 2
  float* G = Xc;
  for (int e = tid; e < l * l; e += nt) {
    const int c1 = e / l, c2 = e % l;
    const float* j1 = Jc + c1 * l;
    const float* j2 = Jc + c2 * l;
    float a = 0.f;
    for (int r = 0; r < l; ++r) a = fmaf(j1[r], j2[r], a);
    G[e] = a;
  }
  __syncthreads();
  for (int e = tid; e < l * l; e += nt) {
    const int c = e / l, r = e % l;  // entry r of column c of W
    float a = 0.f;
    for (int c2 = 0; c2 < l; ++c2) a = fmaf(Jc[c2 * l + r], G[c2 * l + c], a);
    w[(int64_t)r * lp + rank_of[c]] = 1.5f * Jc[c * l + r] - 0.5f * a;
  }
}


// Same algorithm for l <= 128 with every column padded to 128 floats (zeros) so a
// half-warp lane moves its 8 elements of a column with two 16-byte shared-memory
// accesses (float4 index hl and hl + 16), which halves the instructions per pair.
constexpr int kVecL = 128;

__device__ __forceinline__ void ld8(const float* col, int hl, float (&v)[8]) {
  const float4 a = reinterpret_cast<const float4*>(col)[hl];
  const float4 b = reinterpret_cast<const float4*>(col)[hl + 16];
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void st8(float* col, int hl, const float (&v)[8]) {
  reinterpret_cast<float4*>(col)[hl] = make_float4(v[0], v[1], v[2], v[3]);
  reinterpret_cast<float4*>(col)[hl + 16] = make_float4(v[4], v[5], v[6], v[7]);
}

__device__ __forceinline__ void rotate8(float (&u)[8], float (&v)[8], float sn, float tau) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float uu = u[i], vv = v[i];
    u[i] = uu - sn * fmaf(tau, uu, vv);
    v[i] = vv + sn * fmaf(-tau, vv, uu);
  }
}

__global__ void __launch_bounds__(1024) jacobi_vec_kernel(const float* __restrict__ x, int64_t ldx,
                                                          int transposed, int l, int lp,
                                                          float* __restrict__ ut,
                                                          float* __restrict__ s,
                                                          float* __restrict__ w, uint32_t* status,
                                                          uint32_t* info, float tol) {
  extern __shared__ __align__(16) float sm[];
  const int le = l + (l & 1);
  float* Xc = sm;                      // [l][128]
  float* Jc = sm + l * kVecL;          // [l][128]
  float* sig = Jc + l * kVecL;         // [le]
  int* rank_of = reinterpret_cast<int*>(sig + le);
  __shared__ int s_rot;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  const int hw = tid >> 4, hl = tid & 15, nhw = nt >> 4;
  const unsigned hmask = 0xFFFFu << (lane & 16);

  for (int e = tid; e < l * kVecL; e += nt) {
    const int c = e / kVecL, r = e % kVecL;
    Xc[e] = (r < l) ? (transposed ? x[(int64_t)c * ldx + r] : x[(int64_t)r * ldx + c]) : 0.0f;
    Jc[e] = (c == r) ? 1.0f : 0.0f;
  }
  __syncthreads();

  int sweep = 0;
  for (; sweep < kMaxSweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < le - 1; ++round) {
      for (int slot = hw; slot < le / 2; slot += nhw) {
        const int p = rr_player(slot, round, le);
        const int q = rr_player(le - 1 - slot, round, le);
        if (p >= l || q >= l) continue;
        float* xp = Xc + p * kVecL;
        float* xq = Xc + q * kVecL;
        float u[8], v[8];
        ld8(xp, hl, u);
        ld8(xq, hl, v);
        float a = 0.f, b = 0.f, g = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          a = fmaf(u[i], u[i], a);
          b = fmaf(v[i], v[i], b);
          g = fmaf(u[i], v[i], g);
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          a += __shfl_xor_sync(hmask, a, o);
          b += __shfl_xor_sync(hmask, b, o);
          g += __shfl_xor_sync(hmask, g, o);
        }
        if (g == 0.0f || !(fabsf(g) > tol * sqrtf(a * b))) continue;
        const float zeta = __fdividef(b - a, 2.0f * g);
        const float az = fabsf(zeta);
        float t = (az > 1e18f) ? __fdividef(0.5f, az)
                               : __fdividef(1.0f, az + sqrtf(fmaf(az, az, 1.0f)));
        t = copysignf(t, zeta);
        if (zeta == 0.0f) t = 1.0f;
        const float w2 = fmaf(t, t, 1.0f);
        float c = rsqrtf(w2);
        c = c * fmaf(-0.5f * w2, c * c, 1.5f);
        const float sn = c * t;
        const float tau = sn / (1.0f + c);
        if (hl == 0) s_rot = 1;
        rotate8(u, v, sn, tau);
        st8(xp, hl, u);
        st8(xq, hl, v);
        float* jp = Jc + p * kVecL;
        float* jq = Jc + q * kVecL;
        ld8(jp, hl, u);
        ld8(jq, hl, v);
        rotate8(u, v, sn, tau);
        st8(jp, hl, u);
        st8(jq, hl, v);
      }
      __syncthreads();
    }
    const int rot = s_rot;
    __syncthreads();
    if (!rot) break;
  }
  if (tid == 0) {
    if (sweep == kMaxSweeps) set_status(status, ST_JACOBI_NOCONV);
    if (info) atomicMax(info, (uint32_t)(sweep + 1));
  }

  for (int c = warp; c < l; c += nw) {
    float a = 0.f;
    for (int e = lane; e < l; e += 32) a = fmaf(Xc[c * kVecL + e], Xc[c * kVecL + e], a);
    a = warp_sum(a);
    if (lane == 0) sig[c] = sqrtf(a);
  }
  __syncthreads();
  for (int e = tid; e < lp * lp; e += nt) {
    const int r = e / lp, c = e % lp;
    if (r >= l || c >= l) { ut[e] = 0.0f; w[e] = 0.0f; }
  }
  for (int c = warp; c < l; c += nw) {
    const float sc = sig[c];
    int rank = 0;
    for (int c2 = lane; c2 < l; c2 += 32) {
      const float s2 = sig[c2];
      rank += (s2 > sc || (s2 == sc && c2 < c)) ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
    const float inv = sc > 0.0f ? 1.0f / sc : 0.0f;
    for (int e = lane; e < l; e += 32) ut[(int64_t)e * lp + rank] = Xc[c * kVecL + e] * inv;
    if (lane == 0) {
      s[rank] = sc;
      rank_of[c] = rank;
    }
  }
  __syncthreads();
  // Newton-Schulz polish of the accumulated rotations, G = J^T J in X's space
  float* G = Xc;
  for (int e = tid; e < l * l; e += nt) {
    const int c1 = e / l, c2 = e % l;
    const float* j1 = Jc + c1 * kVecL;
    const float* j2 = Jc + c2 * kVecL;
    float a = 0.f;
    for (int r = 0; r < l; ++r) a = fmaf(j1[r], j2[r], a);
    G[e] = a;
  }
  __syncthreads();
  for (int e = tid; e < l * l; e += nt) {
    const int c = e / l, r = e % l;
    float a = 0.f;
    for (int c2 = 0; c2 < l; ++c2) a = fmaf(Jc[c2 * kVecL + r], G[c2 * l + c], a);
    w[(int64_t)r * lp + rank_of[c]] = 1.5f * Jc[c * kVecL + r] - 0.5f * a;
  }
}

size_t jacobi_vec_smem_bytes(int l) {
  return (size_t)(2 * l * kVecL + 2 * l + 4) * sizeof(float);
}

}  // namespace

cudaError_t prepare_jacobi() {
  cudaError_t e = cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)jacobi_smem_bytes(kMaxJacobiL));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(jacobi_vec_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)jacobi_vec_smem_bytes(kVecL));
}

size_t jacobi_smem_bytes(int l) { return (size_t)(2 * l * l + 2 * l + 4) * sizeof(float); }

cudaError_t launch_jacobi_svd(const float* x, int64_t ldx, int transposed, int l, int lp, float* ut,
                              float* s, float* w, float* scratch, uint32_t* status,
                              uint32_t* info, cudaStream_t st, int variant) {
  // the cluster kernel is faster from a few dozen columns on (about 2x at l = 110)
  if (variant == 2 || (variant == 0 && l >= 48))
    return launch_jacobi_cluster(x, ldx, transposed, l, lp, ut, s, w, scratch, status, info, st);
  if (l > kMaxJacobiL) return cudaErrorInvalidValue;
  const size_t smem = jacobi_smem_bytes(l);
  // a pair counts as orthogonal below 8 sqrt(l) u: above the float32 rounding floor of
  // a computed dot product (a few u sqrt(l)), so the sweeps terminate, and small enough
  // that U is orthonormal to ~5e-6 at l ~ 100
  const float tol = 8.0f * sqrtf((float)l) * kEpsF32;
  if (l <= kVecL) {
    jacobi_vec_kernel<<<1, 1024, jacobi_vec_smem_bytes(l), st>>>(x, ldx, transposed, l, lp, ut, s,
                                                                 w, status, info, tol);
    return cudaGetLastError();
  }
  jacobi_kernel<<<1, 1024, smem, st>>>(x, ldx, transposed, l, lp, ut, s, w, status, info, tol);
  return cudaGetLastError();
}

cudaError_t launch_jacobi_svd_pair(const float* x, const float* x_b, int64_t ldx, int transposed, int l,
                                   int lp, float* ut, float* ut_b, float* s, float* s_b, float* w,
                                   float* w_b, float* scratch, float* scratch_b, uint32_t* status,
                                   uint32_t* info, cudaStream_t st, int variant) {
  if (variant == 2 || (variant == 0 && l >= 48))
    return launch_jacobi_cluster(x, ldx, transposed, l, lp, ut, s, w, scratch, status, info, st, x_b,
                                 ut_b, s_b, w_b, scratch_b);
  cudaError_t e = launch_jacobi_svd(x, ldx, transposed, l, lp, ut, s, w, scratch, status, info, st, variant);
  if (e != cudaSuccess) return e;
  return launch_jacobi_svd(x_b, ldx, transposed, l, lp, ut_b, s_b, w_b, scratch_b, status, info, st, variant);
}

}  // namespace rsvd
