// Tensor-core passes over A (Algorithm 4.4 steps 2, 4, 5 and Algorithm 5.1
// step 1) for a bfloat16 A: Y = A X or Y = A^T X, bfloat16 products with
// float32 accumulation in tensor memory.
//
// Shapes: every MMA is M = 128 rows of the output by N = the basis width
// (lp, or 2 lp when the operand carries a hi and a lo half that the epilogue
// sums) by K = 16.  The M side is always A:
//   Y = A X   : A tile = 128 rows x 64 columns of A, K-major (row-major A),
//   Y = A^T X : A tile = 64 rows x 128 columns of A, read as the transposed
//               operand (MN-major), two 64-column TMA boxes.
// The operand X is stored transposed (lp x K, K contiguous, bfloat16) so that
// it is a K-major B operand in both passes.  All tiles are TMA loads with the
// 128-byte swizzle; no multicast.
//
// Work split ("stream-K"): the iterations (row tile t, k tile kk) are laid out
// t-major and cut into gridDim.x equal ranges, one per CTA (one CTA per SM).
// A row tile covered by one CTA is written straight to Y.  A tile split
// between CTAs is finished by the CTA that holds its first k tile (it reaches
// the tile last): the other contributors write their partial sums to a slot
// and raise a flag, and the finishing CTA adds them in CTA order
// (deterministic) and clears the flags.
//
// Warp roles (64 + 128 TM CH threads): warp 0 issues TMA, warp 1 owns tensor memory
// and issues the MMAs from one thread, the 4 TM CH warps from 2 on drain the
// accumulators (each warp reads the 32 TMEM lanes its index allows; with CH = 2 two
// warps share those lanes and take half of the columns each).  With TM = 2 a work unit
// is two 128-row tiles that share every X tile (two MMAs per k step into two
// accumulators), which halves the operand's re-reads from L2.  Every wait is bounded;
// on expiry the kernel records a timeout in the status word and winds down.
//
// Accumulation: the tensor cores add each k16 product into the float32 accumulator
// with truncation, so a long chain of MMAs into one accumulator drifts towards zero
// (about -2e-5 relative over K = 16384, i.e. a thousand k16 steps).  The MMAs of a row
// tile are therefore cut into chunks of kChunkSteps k16 steps, each into a fresh
// accumulator (double-buffered), and the epilogue adds the chunks in registers with IEEE
// float32 additions: the drift then stays that of one chunk.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "sketch_tc.cuh"
#include "tc_ptx.cuh"

namespace rsvd {
namespace {

using namespace tcx;
constexpr int kThreads = 192;   // TM = 1, CH = 1
template <int TM, int CH = 1>
constexpr int threads_for() { return 64 + 128 * TM * CH; }
// k16 accumulation steps per tensor-memory chunk: 128 steps drift by about -2e-6 relative
// (16 k tiles of BK = 64 when every k16 step also adds the residual of A, else 32); halving
// the chunk halves the drift and costs about 4 % more time per pass (drains every 8 k tiles).
constexpr int kChunkSteps = 128;
constexpr int kAccRegs = 128;   // accumulator columns an epilogue thread holds in registers
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int NT>
__device__ __forceinline__ void epi_bar() {  // the epilogue warps only (NT threads)
  asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}
// A barrier of the epilogue warps that also ANDs a flag over them, so that after a bounded
// wait gave up in one warp every epilogue warp takes the same path (no named barrier is
// then left waiting for warps that have stopped).
template <int NT>
__device__ __forceinline__ bool epi_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(NT)
      : "memory");
  return r != 0;
}

struct Range {
  int64_t total;
  int grid;
  __device__ __forceinline__ int64_t start(int c) const { return (int64_t)c * total / grid; }
  __device__ __forceinline__ int cta_of(int64_t it) const {
    int c = (int)(it * grid / total);
    while (c + 1 < grid && start(c + 1) <= it) ++c;
    while (c > 0 && start(c) > it) --c;
    return c;
  }
};

// HILO (one row tile per unit): A arrives as a bfloat16 hi part (map_a) and the bfloat16
// residual lo = A - hi (map_alo, the same tile shape and major-ness); each stage carries
// both tiles and the MMAs of the lo tile accumulate into the same tensor-memory
// accumulator, so the pass sees A to about 16 significant bits.
template <int MODE, int HILO = 0, int TM = 1, int CH = 1, int KB = 1>
__global__ void __launch_bounds__(64 + 128 * TM * CH, 1)
    sketch_tc_kernel(const __grid_constant__ CUtensorMap map_a,
                     const __grid_constant__ CUtensorMap map_alo,
                     const __grid_constant__ CUtensorMap map_x, float* __restrict__ y, int lp,
                     int64_t M, int kt, int64_t total, int n_total, int fold, int lo_off, int stages,
                     float* __restrict__ slots, uint32_t* __restrict__ flags, uint32_t* status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar_full[16], bar_empty[16], bar_acc_full[2], bar_acc_empty[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Range rg{total, (int)gridDim.x};
  const int cta = blockIdx.x;
  const int64_t it0 = rg.start(cta), it1 = rg.start(cta + 1);

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  static_assert(TM == 1 || !HILO, "the residual of A is read with single tiles");
  static_assert(TM * CH <= 2, "at most eight epilogue warps");
  // a k step of a stage is KB adjacent boxes of BK columns (KB = 2: fewer, larger stages)
  constexpr int kChunk = kChunkSteps / ((KB * BK / 16) * (HILO ? 2 : 1));   // k steps per chunk
  constexpr int kEpi = 128 * TM * CH;   // epilogue threads
  constexpr uint32_t a_box = TM * BM * BK * 2 * (HILO ? 2 : 1);  // 16 KB per A tile and box
  constexpr uint32_t a_bytes = KB * a_box;
  const uint32_t x_box = (uint32_t)n_total * BK * 2;
  const uint32_t x_bytes = KB * x_box;
  const uint32_t stage_bytes = a_bytes + x_bytes;
  // A split operand wider than one MMA (2 lp > 256: hi rows from 0, lo rows from 256) is
  // summed by the tensor cores: both MMAs accumulate into the same lp columns.  A narrower
  // one is one MMA of N = 2 lp whose halves the epilogue adds.
  const bool fold_mma = fold && n_total > 256;
  // two accumulators when they fit tensor memory (512 columns): the MMAs of the next chunk
  // then run while the epilogue drains the previous one
  const uint32_t acc_cols = fold_mma ? 256u : (uint32_t)((n_total + 31) & ~31);
  const uint32_t unit_cols = (uint32_t)TM * acc_cols;   // the accumulators of one work unit
  const int nacc = (2 * unit_cols <= 512) ? 2 : 1;
  uint32_t tmem_cols = 32;
  while (tmem_cols < unit_cols * nacc) tmem_cols <<= 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&bar_full[s], 1);
      mbar_init(&bar_empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&bar_acc_full[a], 1);
      mbar_init(&bar_acc_empty[a], 4 * TM * CH);
    }
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_a)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_x)) : "memory");
    if (HILO)
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_alo)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  volatile int* abort_flag = &s_abort;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      // A is streamed once per pass; the operand tiles are read again by every row tile
      const uint64_t pol_a = l2_evict_first_policy(), pol_x = l2_evict_last_policy();
      // the A tiles (both halves with TM = 2, and the residual with HILO) and the operand
      // tile of iteration `it` into stage s
      auto load_a = [&](int64_t it, int s) {
        uint64_t* bar = &bar_full[s];
        const int t = (int)(it / kt), kk = (int)(it % kt);
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) {
          uint8_t* sa = smem + (size_t)s * stage_bytes + kb * a_box;
          const int kx = (kk * KB + kb) * BK;
          if (MODE == 0) {
#pragma unroll
            for (int h = 0; h < TM; ++h)
              tma_load_2d_hint(sa + h * 16384, &map_a, bar, kx, (t * TM + h) * BM, pol_a);
            if (HILO) tma_load_2d_hint(sa + 16384, &map_alo, bar, kx, t * BM, pol_a);
          } else {
#pragma unroll
            for (int h = 0; h < TM; ++h) {
              tma_load_2d_hint(sa + h * 16384, &map_a, bar, (t * TM + h) * BM, kx, pol_a);
              tma_load_2d_hint(sa + h * 16384 + 8192, &map_a, bar, (t * TM + h) * BM + 64, kx, pol_a);
            }
            if (HILO) {
              tma_load_2d_hint(sa + 16384, &map_alo, bar, t * BM, kx, pol_a);
              tma_load_2d_hint(sa + 16384 + 8192, &map_alo, bar, t * BM + 64, kx, pol_a);
            }
          }
        }
      };
      auto load_x = [&](int64_t it, int s) {
        const int kk = (int)(it % kt);
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) {
          uint8_t* sx = smem + (size_t)s * stage_bytes + a_bytes + (size_t)kb * x_box;
          for (int c = 0; c * 256 < n_total; ++c)
            tma_load_2d_hint(sx + (size_t)c * 256 * 128, &map_x, &bar_full[s], (kk * KB + kb) * BK, c * 256,
                             pol_x);
        }
      };
      // A is an input of the whole call and is never written by it: the A tiles of the
      // first stages go out before waiting for the launch that wrote the operand.
      const int64_t npre = (it1 - it0 < stages) ? it1 - it0 : stages;
      for (int64_t j = 0; j < npre; ++j) {
        mbar_expect_tx(&bar_full[j], stage_bytes);
        load_a(it0 + j, (int)j);
      }
      pdl_wait();
      for (int64_t j = 0; j < npre; ++j) load_x(it0 + j, (int)j);
      int64_t i = npre;
      for (int64_t it = it0 + npre; it < it1; ++it, ++i) {
        const int s = (int)(i % stages);
        const uint32_t ph = (uint32_t)((i / stages) & 1);
        if (!mbar_wait(&bar_empty[s], ph ^ 1u, abort_flag, status)) break;
        mbar_expect_tx(&bar_full[s], stage_bytes);
        load_a(it, s);
        load_x(it, s);
      }
      // let the copies still in flight land before the CTA can exit
      const int64_t issued = i;
      for (int64_t j = (issued > stages ? issued - stages : 0); j < issued; ++j) {
        const int s = (int)(j % stages);
        const uint32_t ph = (uint32_t)((j / stages) & 1);
        for (uint32_t w = 0; w < kSpinLimit && !mbar_try_wait(&bar_full[s], ph); ++w) __nanosleep(64);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc_full = instr_desc(n_total < 256 ? n_total : 256, MODE);
      const uint32_t idesc_tail = instr_desc(n_total > 256 ? n_total - 256 : 16, MODE);
      int64_t i = 0;
      int ch = 0;   // chunk counter: accumulator buffer ch % nacc, phase (ch / nacc) & 1
      bool ok = true;
      for (int64_t it = it0; it < it1 && ok;) {
        const int t = (int)(it / kt);
        const int64_t seg_end = min(it1, (int64_t)(t + 1) * kt);
        for (; it < seg_end && ok; ++ch) {
          const int64_t ch_begin = it, ch_end = min(seg_end, it + kChunk);
          const int ab = ch % nacc;
          const uint32_t acc = tmem + (uint32_t)ab * unit_cols;
          if (!mbar_wait(&bar_acc_empty[ab], ((uint32_t)(ch / nacc) & 1u) ^ 1u, abort_flag, status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          for (; it < ch_end; ++it, ++i) {
            const int s = (int)(i % stages);
            const uint32_t ph = (uint32_t)((i / stages) & 1);
            if (!mbar_wait(&bar_full[s], ph, abort_flag, status)) { ok = false; break; }
            tc_fence_after();
            const uint32_t sa0 = smem_u32(smem + (size_t)s * stage_bytes);
            const bool first = (it == ch_begin);
#pragma unroll
            for (int kb = 0; kb < KB; ++kb) {
            const uint32_t sa = sa0 + kb * a_box;
            const uint32_t sx = sa0 + a_bytes + kb * x_box;
#pragma unroll
            for (int j = 0; j < BK / 16; ++j) {
#pragma unroll
              for (int h = 0; h < TM; ++h) {
                uint64_t adesc;
                if (MODE == 0)
                  adesc = smem_desc(sa + h * 16384 + j * 32, 16, 1024);       // K-major: +32 B per k16
                else
                  adesc = smem_desc(sa + h * 16384 + j * 2048, 8192, 1024);   // MN-major: +16 rows of 128 B
                for (int c = 0; c * 256 < n_total; ++c) {
                  const uint64_t bdesc = smem_desc(sx + c * 256 * 128 + j * 32, 16, 1024);
                  const uint32_t idesc = (c == 0) ? idesc_full : idesc_tail;
                  const uint32_t dcol = fold_mma ? 0u : (uint32_t)c * 256;
                  const uint32_t accum = (first && kb == 0 && j == 0 && (c == 0 || !fold_mma)) ? 0u : 1u;
                  mma_bf16(acc + h * acc_cols + dcol, adesc, bdesc, idesc, accum);
                  if (HILO) {
                    const uint64_t adesc_lo = MODE == 0 ? smem_desc(sa + 16384 + j * 32, 16, 1024)
                                                        : smem_desc(sa + 16384 + j * 2048, 8192, 1024);
                    mma_bf16(acc + dcol, adesc_lo, bdesc, idesc, 1u);
                  }
                }
              }
            }
            }
            mma_commit(&bar_empty[s]);
          }
          if (ok) mma_commit(&bar_acc_full[ab]);
        }
      }
    }
  } else {
    // ---------------- epilogue (warps 2 .. 1 + 4 TM CH) ----------------
    const int quad = warp & 3;
    const int idx = (warp - 2) >> 2;
    const int half = TM == 2 ? idx : 0;   // which 128-row tile of the unit
    const int chalf = CH == 2 ? idx : 0;  // which half of the columns
    const int row = half * BM + quad * 32 + lane;
    // this thread's columns: [cb, cb + ncols), multiples of 16 (lp is a multiple of 16)
    const int cmid = CH == 2 ? (int)(((lp >> 1) + 15) & ~15) : lp;
    const int cb = chalf ? cmid : 0;
    const int ncols = chalf ? lp - cmid : cmid;
    const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)half * acc_cols + (uint32_t)cb;
    const bool fold_epi = fold && !fold_mma;
    float racc[kAccRegs];
    int ch = 0;
    for (int64_t it = it0; it < it1;) {
      const int t = (int)(it / kt);
      const int64_t tile_b = (int64_t)t * kt, tile_e = tile_b + kt;
      const int64_t seg_end = min(it1, tile_e);
      const int c_first = rg.cta_of(tile_b), c_last = rg.cta_of(tile_e - 1);
      bool ok = true;
      // drain the chunks of this segment into registers (IEEE float32 additions)
      for (int64_t cs = it; cs < seg_end; cs = min(seg_end, cs + kChunk), ++ch) {
        ok = __all_sync(0xffffffffu, mbar_wait(&bar_acc_full[ch % nacc], (uint32_t)(ch / nacc) & 1u,
                                               abort_flag, status));
        tc_fence_after();
        const uint32_t tb = tbase + (uint32_t)(ch % nacc) * unit_cols;
        const bool first = (cs == it);
#pragma unroll
        for (int c0 = 0; c0 < kAccRegs; c0 += 16) {   // 16 columns at a time (ncols % 16 == 0)
          if (c0 < ncols) {
            float v[16];
            tmem_ld16(tb + c0, v);
            if (fold_epi) {
              float w2[16];
              tmem_ld16(tb + lo_off + c0, w2);
#pragma unroll
              for (int q = 0; q < 16; ++q) v[q] += w2[q];
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) racc[c0 + q] = first ? v[q] : racc[c0 + q] + v[q];
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar_acc_empty[ch % nacc]);
        if (!ok) break;
      }
      ok = epi_all<kEpi>(ok);
      const int64_t grow = (int64_t)t * (BM * TM) + row;
      const bool valid_row = grow < M;
      const bool direct = (c_first == c_last);
      const bool finisher = !direct && (cta == c_first);
      if (finisher && ok) {
        // wait until every later contributor has published its partial sum
        for (int c = c_first + 1; c <= c_last; ++c) {
          uint32_t w = 0;
          while (ld_acquire(flags + c) == 0u) {
            if (++w > kSpinLimit || *abort_flag) {
              set_status(status, ST_TIMEOUT);
              *abort_flag = 1;
              break;
            }
            __nanosleep(128);
          }
        }
      }
      if (ok && valid_row) {
#pragma unroll
        for (int c0 = 0; c0 < kAccRegs; c0 += 32) {
          if (c0 < ncols) {
            const int nc = min(32, ncols - c0);
            const int col = cb + c0;
            if (direct || finisher) {
              if (finisher) {
                for (int c = c_first + 1; c <= c_last; ++c) {
                  const float4* src =
                      reinterpret_cast<const float4*>(slots + ((size_t)c * BM * TM + row) * lp + col);
#pragma unroll
                  for (int q = 0; q < 32; q += 4) {
                    if (q < nc) {
                      const float4 w4 = src[q >> 2];
                      racc[c0 + q] += w4.x; racc[c0 + q + 1] += w4.y;
                      racc[c0 + q + 2] += w4.z; racc[c0 + q + 3] += w4.w;
                    }
                  }
                }
              }
              float* dst = y + grow * lp + col;
#pragma unroll
              for (int q = 0; q < 32; q += 4)
                if (q < nc)
                  *reinterpret_cast<float4*>(dst + q) =
                      make_float4(racc[c0 + q], racc[c0 + q + 1], racc[c0 + q + 2], racc[c0 + q + 3]);
            } else {
              float4* dst = reinterpret_cast<float4*>(slots + ((size_t)cta * BM * TM + row) * lp + col);
#pragma unroll
              for (int q = 0; q < 32; q += 4)
                if (q < nc)
                  dst[q >> 2] = make_float4(racc[c0 + q], racc[c0 + q + 1], racc[c0 + q + 2], racc[c0 + q + 3]);
            }
          }
        }
      }
      if (!direct && !finisher) {
        // publish this CTA's partial of tile t (its first segment)
        __threadfence();
        epi_bar<kEpi>();
        if (warp == 2 && lane == 0) st_release(flags + cta, 1u);
      } else if (finisher) {
        epi_bar<kEpi>();  // all rows have read the partials
        if (warp == 2 && lane == 0)
          for (int c = c_first + 1; c <= c_last; ++c) flags[c] = 0u;
      }
      it = seg_end;
      if (!ok) break;
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tmem_cols)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------


struct TcBuffers {
  float* slots = nullptr;
  uint32_t* flags = nullptr;
  int grid = 0;
};

size_t smem_bytes(int n_total, int stages, int a_tiles = 1, int kb = 1) {
  return (size_t)stages * kb * ((size_t)a_tiles * BM * BK * 2 + (size_t)n_total * BK * 2) + 1024;
}

// Widest operand (columns) for which a work unit takes two row tiles: two double-buffered
// accumulators of 128 columns fill the 512 columns of tensor memory.
constexpr int kPairMaxN = 128;

constexpr int kStageBudget = 200 * 1024;
constexpr int kPassSmemCap = kStageBudget + 4096;   // stages plus the 1 KB alignment pad

int pick_stages(int n_total, int a_tiles = 1, int kb = 1) {
  const size_t budget = kStageBudget;
  int s = (int)(budget / (kb * ((size_t)a_tiles * BM * BK * 2 + (size_t)n_total * BK * 2)));
  if (s > 8) s = 8;
  return s < 2 ? 2 : s;
}

}  // namespace

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static int get_encoder() {
  if (g_encode) return 0;
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return -1;
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return 0;
}

// 2-D bfloat16 tensor map: inner dimension `inner` (contiguous), `outer` rows
// of `ld` elements, box {box_inner, box_outer}, 128-byte swizzle.
int tc_encode_2d(void* map, const void* base, uint64_t inner, uint64_t outer, uint64_t ld,
              uint32_t box_inner, uint32_t box_outer) {
  if (get_encoder()) return -1;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {ld * 2};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                        const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -1;
}

int64_t tc_ld(int64_t k) { return round_up(k, 8); }
int tc_lo_offset(int lp) { return 2 * lp <= 256 ? lp : 256; }
static int fold_ntotal(int lp) { return 2 * lp <= 256 ? 2 * lp : 512; }

int tc_plan_init(TcPlan* tc, int64_t m, int64_t n, int64_t lda, int lp, __nv_bfloat16* xbf,
                 int num_sms) {
  tc->m = m;
  tc->n = n;
  tc->lda = lda;
  tc->lp = lp;
  tc->num_sms = num_sms;
  tc->xbf = xbf;
  tc->a_bound = nullptr;
  if (lp > 256 || lp % 16) return -1;
  const int64_t ldn = tc_ld(n), ldm = tc_ld(m);
  if (tc_encode_2d(tc->map_x_n, xbf, n, lp, ldn, BK, lp)) return -1;
  if (tc_encode_2d(tc->map_x_t, xbf, m, lp, ldm, BK, lp)) return -1;
  const int nf = fold_ntotal(lp);
  if (tc_encode_2d(tc->map_x_t2, xbf, m, tc_lo_offset(lp) + lp, ldm, BK, nf > 256 ? 256 : nf)) return -1;
  if (tc_encode_2d(tc->map_x_n2, xbf, n, tc_lo_offset(lp) + lp, ldn, BK, nf > 256 ? 256 : nf)) return -1;
  TcBuffers* b = new TcBuffers();
  b->grid = num_sms;
  if (cudaMalloc(&b->slots, sizeof(float) * (size_t)num_sms * 2 * BM * lp) != cudaSuccess ||
      cudaMalloc(&b->flags, sizeof(uint32_t) * (size_t)num_sms) != cudaSuccess ||
      cudaMemset(b->flags, 0, sizeof(uint32_t) * (size_t)num_sms) != cudaSuccess) {
    cudaGetLastError();
    if (b->slots) cudaFree(b->slots);
    if (b->flags) cudaFree(b->flags);
    delete b;
    return -1;
  }
  tc->priv = b;
  // One limit for every pass kernel, above the stage budget of pick_stages: the attribute
  // belongs to the kernel, not to this plan, so a later plan must not lower it under an
  // earlier one.
  for (const void* fn : {(const void*)sketch_tc_kernel<0>, (const void*)sketch_tc_kernel<1>,
                         (const void*)sketch_tc_kernel<1, 1>, (const void*)sketch_tc_kernel<0, 1>,
                         (const void*)sketch_tc_kernel<0, 0, 2>,
                         (const void*)sketch_tc_kernel<1, 0, 2>,
                         (const void*)sketch_tc_kernel<0, 0, 1, 2>,
                         (const void*)sketch_tc_kernel<1, 0, 1, 2>,
                         (const void*)sketch_tc_kernel<0, 1, 1, 2>,
                         (const void*)sketch_tc_kernel<1, 1, 1, 2>,
                         (const void*)sketch_tc_kernel<0, 0, 1, 1, 2>,
                         (const void*)sketch_tc_kernel<1, 0, 1, 1, 2>,
                         (const void*)sketch_tc_kernel<1, 1, 1, 1, 2>,
                         (const void*)sketch_tc_kernel<0, 1, 1, 1, 2>,
                         (const void*)sketch_tc_kernel<0, 0, 2, 1, 2>,
                         (const void*)sketch_tc_kernel<1, 0, 2, 1, 2>,
                         (const void*)sketch_tc_kernel<0, 0, 1, 2, 2>,
                         (const void*)sketch_tc_kernel<1, 0, 1, 2, 2>,
                         (const void*)sketch_tc_kernel<0, 1, 1, 2, 2>,
                         (const void*)sketch_tc_kernel<1, 1, 1, 2, 2>})
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kPassSmemCap) !=
        cudaSuccess)
      return -1;
  tc->ready = true;
  return 0;
}

int tc_bind_a(TcPlan* tc, const void* A, int with_lo) {
  if (!tc->ready) return -1;
  if (A == tc->a_bound && with_lo == tc->lo_bound) return 0;
  if (reinterpret_cast<uintptr_t>(A) & 15) return -1;
  if (tc_encode_2d(tc->map_a_n, A, tc->n, tc->m, tc->lda, BK, BM)) return -1;
  if (tc_encode_2d(tc->map_a_t, A, tc->n, tc->m, tc->lda, 64, BK)) return -1;
  if (with_lo) {
    const __nv_bfloat16* lo = static_cast<const __nv_bfloat16*>(A) + tc->m * tc->lda;
    if (tc_encode_2d(tc->map_a_lo, lo, tc->n, tc->m, tc->lda, 64, BK)) return -1;
    if (tc_encode_2d(tc->map_a_lo_n, lo, tc->n, tc->m, tc->lda, BK, BM)) return -1;
  }
  tc->a_bound = A;
  tc->lo_bound = with_lo;
  return 0;
}

int tc_pass(TcPlan* tc, int trans, int split_x, int hilo, float* out, int* splits,
            cudaStream_t st) {
  if (!tc->ready || !tc->a_bound) return -1;
  if (hilo && !tc->lo_bound) return -1;
  TcBuffers* b = static_cast<TcBuffers*>(tc->priv);
  const int lp = tc->lp;
  const int n_total = split_x ? fold_ntotal(lp) : lp;
  const int lo_off = split_x ? tc_lo_offset(lp) : 0;
  const int64_t M = trans ? tc->n : tc->m;
  const int64_t K = trans ? tc->m : tc->n;
  // two row tiles per work unit while both accumulators stay double-buffered
  const int tm = (!hilo && n_total <= kPairMaxN) ? 2 : 1;
  const int at = hilo ? 2 : tm;   // A tiles per box
  // operands wider than 128 columns: two adjacent boxes along k per stage when two such
  // stages fit the budget (half the stages and barrier round trips for the same bytes in
  // flight; measured 6 % faster at l_p = 256, while at l_p = 112 the deeper ring of single
  // boxes is faster)
  const size_t box_set = (size_t)at * BM * BK * 2 + (size_t)n_total * BK * 2;
  const int kb = (n_total > kPairMaxN && 4 * box_set <= (size_t)kStageBudget) ? 2 : 1;
  const int kt = (int)cdiv(K, (int64_t)BK * kb);
  const int64_t total = cdiv(M, (int64_t)BM * tm) * kt;
  const int grid = (int)(total < b->grid ? total : b->grid);
  const int stages = pick_stages(n_total, at, kb);
  const size_t sm = smem_bytes(n_total, stages, at, kb);
  const CUtensorMap* ma = reinterpret_cast<const CUtensorMap*>(trans ? tc->map_a_t : tc->map_a_n);
  const CUtensorMap* malo = reinterpret_cast<const CUtensorMap*>(
      hilo ? (trans ? tc->map_a_lo : tc->map_a_lo_n) : (trans ? tc->map_a_t : tc->map_a_n));
  const CUtensorMap* mx = reinterpret_cast<const CUtensorMap*>(
      trans ? (split_x ? tc->map_x_t2 : tc->map_x_t) : (split_x ? tc->map_x_n2 : tc->map_x_n));
  // launched as a programmatic dependent: the A tiles of the first stages are loaded
  // while the launch that converts the operand finishes.  Bases wider than kAccRegs
  // columns take two epilogue warps per TMEM lane quarter (CH = 2), each holding half of
  // a row's columns in registers.
  const int ch = lp > kAccRegs ? 2 : 1;
  auto go = [&](auto kernel, int threads) {
    return launch_pdl(kernel, dim3(grid), dim3(threads), sm, st, *ma, *malo, *mx, out, lp, M, kt,
                      total, n_total, split_x, lo_off, stages, b->slots, b->flags, tc->status);
  };
  cudaError_t e;
#define RSVD_PASS(MO, HI, T, C)                                                            \
  e = (kb == 2) ? go(sketch_tc_kernel<MO, HI, T, C, 2>, threads_for<T, C>())               \
                : go(sketch_tc_kernel<MO, HI, T, C, 1>, threads_for<T, C>())
  if (ch == 2) {
    if (hilo && trans) RSVD_PASS(1, 1, 1, 2);
    else if (hilo) RSVD_PASS(0, 1, 1, 2);
    else if (trans) RSVD_PASS(1, 0, 1, 2);
    else RSVD_PASS(0, 0, 1, 2);
  } else if (hilo && trans) {
    RSVD_PASS(1, 1, 1, 1);
  } else if (hilo) {
    RSVD_PASS(0, 1, 1, 1);
  } else if (tm == 2 && trans) {
    RSVD_PASS(1, 0, 2, 1);
  } else if (tm == 2) {
    RSVD_PASS(0, 0, 2, 1);
  } else if (trans) {
    RSVD_PASS(1, 0, 1, 1);
  } else {
    RSVD_PASS(0, 0, 1, 1);
  }
#undef RSVD_PASS
  if (e != cudaSuccess) return -1;
  *splits = 1;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int64_t tc_partial_elems(int64_t m, int64_t n, int lp, int num_sms) {
  (void)num_sms;
  return (m > n ? m : n) * (int64_t)lp;
}

void tc_plan_destroy(TcPlan* tc) {
  if (tc->priv) {
    TcBuffers* b = static_cast<TcBuffers*>(tc->priv);
    if (b->slots) cudaFree(b->slots);
    if (b->flags) cudaFree(b->flags);
    delete b;
    tc->priv = nullptr;
  }
  tc->ready = false;
}

}  // namespace rsvd

// ---------------------------------------------------------------------------
// Allocation-free pass (rsvd_sketch_bf16_noalloc)
//
// The same kernel as tc_pass, for callers that cannot allocate device memory.
// Its stream-K scratch -- the partial sums of row tiles that two CTAs share
// and the flags that hand them over -- lives in file-scope device arrays of a
// fixed size (g_noalloc_slots: 152 CTAs x 128 rows x 128 columns of float32,
// 9.5 MiB; g_noalloc_flags: 152 words), which every GPU that loads the library
// keeps until the process exits.  Host code must not hand these symbols to a
// kernel (on the host they are stand-ins, not device addresses): the set-up
// below asks the runtime for their device addresses, once per device.
// ---------------------------------------------------------------------------

#include <mutex>

namespace rsvd {
namespace {

constexpr int kNoAllocMaxCtas = 152;
constexpr int kNoAllocMaxL = 128;

__device__ __align__(256) float g_noalloc_slots[(size_t)kNoAllocMaxCtas * BM * kNoAllocMaxL];
__device__ __align__(256) uint32_t g_noalloc_flags[kNoAllocMaxCtas];

struct NoAllocDevice {
  bool ready = false;
  float* slots = nullptr;
  uint32_t* flags = nullptr;
  int num_sms = 0;
};

constexpr int kNoAllocMaxDevices = 64;
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];
std::mutex g_noalloc_mu;

// Once per device, with that device current: device addresses of the scratch
// arrays, the SM count, and the shared-memory limit of both kernel variants.
int noalloc_setup(int dev, NoAllocDevice** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return -1;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoAllocDevice& d = g_noalloc_dev[dev];
  if (!d.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_slots) != cudaSuccess) return -1;
    d.slots = static_cast<float*>(p);
    if (cudaGetSymbolAddress(&p, g_noalloc_flags) != cudaSuccess) return -1;
    d.flags = static_cast<uint32_t*>(p);
    if (cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return -1;
    // the same limit as the plans set (never lower it under a live plan)
    if (cudaFuncSetAttribute(sketch_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kPassSmemCap) != cudaSuccess ||
        cudaFuncSetAttribute(sketch_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kPassSmemCap) != cudaSuccess)
      return -1;
    d.ready = true;
  }
  *out = &d;
  return 0;
}

}  // namespace
}  // namespace rsvd

extern "C" rsvd_status_t rsvd_sketch_bf16_noalloc(const void* A, int64_t m, int64_t n,
                                                  int64_t lda, int32_t transpose, const void* Xt,
                                                  int64_t ldxt, int32_t l, float* Y,
                                                  uint32_t* status, void* stream) {
  using namespace rsvd;
  if (!A || !Xt || !Y || m < 1 || n < 1) return RSVD_ERR_INVALID_ARG;
  if (l < 16 || l > kNoAllocMaxL || l % 16 != 0) return RSVD_ERR_INVALID_ARG;
  const int64_t K = transpose ? m : n;
  if (lda < n || lda % 8 != 0 || ldxt < K || ldxt % 8 != 0) return RSVD_ERR_INVALID_ARG;
  // TMA reads A and Xt from 16-byte boundaries; the epilogue writes Y as float4
  if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(Xt) & 15) ||
      (reinterpret_cast<uintptr_t>(Y) & 15))
    return RSVD_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RSVD_ERR_CUDA;
  NoAllocDevice* d = nullptr;
  if (noalloc_setup(dev, &d) != 0) return RSVD_ERR_CUDA;
  alignas(64) unsigned char map_a[128];
  alignas(64) unsigned char map_x[128];
  if (tc_encode_2d(map_a, A, n, m, lda, BK, transpose ? 64 : BM)) return RSVD_ERR_CUDA;
  if (tc_encode_2d(map_x, Xt, K, l, ldxt, BK, l)) return RSVD_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t M = transpose ? n : m;
  const int kt = (int)cdiv(K, BK);
  const int64_t total = cdiv(M, BM) * kt;
  int grid = d->num_sms < kNoAllocMaxCtas ? d->num_sms : kNoAllocMaxCtas;
  if (total < grid) grid = (int)total;
  // the flags must start at zero (the kernel clears the ones it consumes, but a
  // call that gave up on a wait can leave some set)
  if (cudaMemsetAsync(d->flags, 0, sizeof(uint32_t) * kNoAllocMaxCtas, st) != cudaSuccess)
    return RSVD_ERR_CUDA;
  const int stages = pick_stages(l);
  const size_t sm = smem_bytes(l, stages);
  const CUtensorMap* ma = reinterpret_cast<const CUtensorMap*>(map_a);
  const CUtensorMap* mx = reinterpret_cast<const CUtensorMap*>(map_x);
  if (transpose)
    sketch_tc_kernel<1><<<grid, kThreads, sm, st>>>(*ma, *ma, *mx, Y, l, M, kt, total, l, 0, 0, stages,
                                                    d->slots, d->flags, status);
  else
    sketch_tc_kernel<0><<<grid, kThreads, sm, st>>>(*ma, *ma, *mx, Y, l, M, kt, total, l, 0, 0, stages,
                                                    d->slots, d->flags, status);
  return cudaGetLastError() == cudaSuccess ? RSVD_OK : RSVD_ERR_CUDA;
}
