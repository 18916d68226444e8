// Placeholder until the tcgen05 kernels land: the tensor-core path reports
// itself unavailable so that plan creation fails with an error.
#include "sketch_tc.cuh"

namespace rsvd {
int tc_plan_init(TcPlan*, int64_t, int64_t, int64_t, int, __nv_bfloat16*, int) { return -1; }
int tc_bind_a(TcPlan*, const void*) { return -1; }
int tc_pass(TcPlan*, int, int, float*, int*, cudaStream_t) { return -1; }
int64_t tc_partial_elems(int64_t, int64_t, int, int) { return 0; }
void tc_plan_destroy(TcPlan*) {}
}  // namespace rsvd
