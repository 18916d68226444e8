// Tensor-core (tcgen05, bfloat16 in / float32 accumulate) passes over A:
// Y = A X and Y = A^T X with A row-major bfloat16 and the operand X stored
// transposed in bfloat16 (lp x K, K contiguous).  Implemented in k_sketch_tc.cu.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rsvd {

struct TcPlan {
  int64_t m = 0, n = 0, lda = 0;
  int lp = 0, num_sms = 0;
  __nv_bfloat16* xbf = nullptr;   // operand buffer, 2 lp x max(m, n)
  const void* a_bound = nullptr;  // A described by the tensor maps below
  alignas(64) unsigned char map_a_n[128];  // A tiles for Y = A X   (K-major operand)
  alignas(64) unsigned char map_a_t[128];  // A tiles for Y = A^T X (MN-major operand)
  alignas(64) unsigned char map_x_n[128];  // X^T tiles, K = n
  alignas(64) unsigned char map_x_t[128];  // X^T tiles, K = m (lp rows)
  alignas(64) unsigned char map_x_t2[128]; // X^T tiles, K = m (hi rows, then lo rows at tc_lo_offset)
  alignas(64) unsigned char map_x_n2[128]; // X^T tiles, K = n (hi rows, then lo rows at tc_lo_offset)
  alignas(64) unsigned char map_a_lo[128]; // residual lo = A - hi, stacked m rows below A (Y = A^T X)
  alignas(64) unsigned char map_a_lo_n[128]; // the same residual as K-major tiles (Y = A X)
  bool ready = false;
  int lo_bound = 0;
  uint32_t* status = nullptr;     // device status word of the owning plan
  void* priv = nullptr;           // stream-K slots and flags
};

// Leading dimension (elements) of the transposed bfloat16 operand for a K extent:
// TMA wants row strides that are multiples of 16 bytes.
int64_t tc_ld(int64_t k);
// Row at which the lo half of a split operand starts (lp when 2 lp <= 256, else 256),
// and the rows the operand buffer needs (lo offset + lp).
int tc_lo_offset(int lp);

// 0 on success.
int tc_plan_init(TcPlan* tc, int64_t m, int64_t n, int64_t lda, int lp, __nv_bfloat16* xbf,
                 int num_sms);
// with_lo: A is followed (m rows of lda further) by its bfloat16 residual lo = A - hi.
int tc_bind_a(TcPlan* tc, const void* A, int with_lo);
// One pass.  trans = 0: Y = A X (X^T is lp x n in xbf); trans = 1: Y = A^T X (X^T is lp x m);
// with split_x = 1 the operand has a hi and a lo half (rows 0 and tc_lo_offset(lp)) whose
// products are summed; hilo = 1 also reads the residual of A.  Writes *splits slabs of (rows x lp) float32 into `partial`.
int tc_pass(TcPlan* tc, int trans, int split_x, int hilo, float* partial, int* splits,
            cudaStream_t st);
// 2-D bfloat16 tensor map, 128-byte swizzle: inner dimension `inner` (contiguous), `outer`
// rows of `ld` elements, box {box_inner, box_outer}.  0 on success.
int tc_encode_2d(void* map, const void* base, uint64_t inner, uint64_t outer, uint64_t ld,
                 uint32_t box_inner, uint32_t box_outer);
int64_t tc_partial_elems(int64_t m, int64_t n, int lp, int num_sms);
void tc_plan_destroy(TcPlan* tc);

}  // namespace rsvd
