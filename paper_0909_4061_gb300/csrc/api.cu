// C ABI of the library: plan creation, argument checks, workspace, and the
// sequence of kernel launches for each entry point of include/rsvd.h.
//
// rsvd_svd (Algorithm 4.4 as Stage A, Algorithm 5.1 + Remark 5.1 as Stage B):
//   Omega            draw (Philox + Box-Muller) or the caller's matrix
//   Y0 = A Omega     pass over A, split-K partials
//   Q0               Cholesky-QR rounds (the first round sums the partials)
//   for j = 1..q:    Yt_j = A^T Q_{j-1} -> Qt_j ;  Y_j = A Qt_j -> Q_j
//   B^T = A^T Q_q    pass over A, then Cholesky-QR rounds B^T = Q_B R_B
//   R_B^T = Ut S W^T one-sided Jacobi in one CTA
//   U = Q_q Ut_k, V = Q_B W_k, S = S_k
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <utility>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "sketch_tc.cuh"

using namespace rsvd;

struct rsvd_plan_s {
  int64_t m = 0, n = 0, lda = 0, maxmn = 0;
  int k = 0, p = 0, q = 0, l = 0, lp = 0;
  uint64_t seed = 0;
  rsvd_options_t opt{};
  cudaStream_t st = nullptr;
  int device = 0, num_sms = kNumSMs;
  int splits_n = 1, splits_t = 1;  // split-K of the passes Y = A X and Y = A^T X (FP32 path)
  int nblk = 1;
  bool omega_user = false;
  // workspace (device)
  float* omega = nullptr;    // n x lp
  float* qbuf = nullptr;     // m x lp   basis Q_j
  float* qtbuf = nullptr;    // n x lp   basis Qt_j, later Q_B
  float* tmp1 = nullptr;     // maxmn x lp
  float* tmp2 = nullptr;     // maxmn x lp
  float* partial = nullptr;  // split-K partial results
  int64_t partial_elems = 0;
  float* gpart = nullptr;    // nblk x lp x lp
  uint8_t* rimg = nullptr;   // bfloat16 planes of R^-1 for the tensor-core apply (l_p > 128)
  float* small = nullptr;    // 24 x lp x lp: g, lbuf, rtmp, rinv, racc, ut, w, scratch, single pass
  float* psi = nullptr;      // m x lp   second test matrix of the single-pass sketch
  float* sig2 = nullptr;     // 2 lp     singular values of X1, X2 (single pass)
  float* sig = nullptr;      // lp
  int* srft_freq = nullptr;  // l / 2 sampled frequencies of the SRFT test matrix
  uint32_t* status = nullptr;
  __nv_bfloat16* xbf = nullptr;  // 2 lp x maxmn: transposed bfloat16 operand of the tensor-core passes
  TcPlan tc{};
  // rsvd_svd_host staging
  void* a_dev = nullptr;
  float* a_f32 = nullptr;  // float32 staging of A for the host_f32 option
  float *u_dev = nullptr, *s_dev = nullptr, *v_dev = nullptr;
  size_t ws_bytes = 0;
  // CUDA graph of rsvd_svd for one (A, U, S, V) binding
  cudaGraphExec_t gexec = nullptr;
  const void* g_a = nullptr;
  const float *g_u = nullptr, *g_s = nullptr, *g_v = nullptr;
  int64_t g_launches[RSVD_NUM_STEPS] = {};
  bool use_graph = true;
  // tracing
  uint32_t prof_mask = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[RSVD_NUM_STEPS];
  int ev_used[RSVD_NUM_STEPS] = {};
  int64_t launches[RSVD_NUM_STEPS] = {};

  float* g() { return small; }
  float* lbuf() { return small + 1 * (size_t)lp * lp; }
  float* rtmp() { return small + 2 * (size_t)lp * lp; }
  float* rinv() { return small + 3 * (size_t)lp * lp; }
  float* racc() { return small + 4 * (size_t)lp * lp; }
  float* ut() { return small + 5 * (size_t)lp * lp; }
  float* w() { return small + 6 * (size_t)lp * lp; }
  float* sq() { return small + 7 * (size_t)lp * lp; }
  // single pass (Section 5.5): 16 more l x l blocks (see stage_single_pass)
  float* sp(int i) { return small + (size_t)(8 + i) * lp * lp; }
};

namespace {

#define TRY(expr)                                 \
  do {                                            \
    cudaError_t _e = (expr);                      \
    if (_e != cudaSuccess) return RSVD_ERR_CUDA;  \
  } while (0)

#define TRYS(expr)                          \
  do {                                      \
    rsvd_status_t _s = (expr);              \
    if (_s != RSVD_OK) return _s;           \
  } while (0)

template <class T>
rsvd_status_t dalloc(rsvd_plan_t P, T** ptr, size_t elems) {
  *ptr = nullptr;
  if (elems == 0) elems = 1;
  const size_t bytes = elems * sizeof(T);
  if (cudaMalloc(reinterpret_cast<void**>(ptr), bytes) != cudaSuccess) {
    cudaGetLastError();
    return RSVD_ERR_ALLOC;
  }
  P->ws_bytes += bytes;
  return RSVD_OK;
}

void free_plan(rsvd_plan_t P) {
  if (!P) return;
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  for (auto& v : P->ev)
    for (auto& e : v) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
  void* bufs[] = {P->omega, P->qbuf, P->qtbuf, P->tmp1, P->tmp2, P->partial, P->gpart,
                  P->small, P->sig,  P->status, P->xbf, P->a_dev, P->u_dev, P->s_dev,
                  P->v_dev, P->srft_freq, P->psi, P->sig2, P->rimg, P->a_f32};
  for (void* b : bufs)
    if (b) cudaFree(b);
  tc_plan_destroy(&P->tc);
  delete P;
}

int choose_splits(int64_t M, int64_t N, int64_t K, int sms) {
  const int64_t tiles = cdiv(M, 128) * cdiv(N, 64);
  const int64_t target = 4LL * sms;
  int64_t s = cdiv(target, tiles);
  const int64_t kmax = std::max<int64_t>(1, cdiv(K, 16) / 8);
  s = std::min<int64_t>(s, kmax);
  s = std::min<int64_t>(s, 32);
  return (int)std::max<int64_t>(s, 1);
}

rsvd_status_t take_status(rsvd_plan_t P) {
  uint32_t st = 0;
  TRY(cudaMemcpyAsync(&st, P->status, sizeof(st), cudaMemcpyDeviceToHost, P->st));
  TRY(cudaStreamSynchronize(P->st));
  if (st) TRY(cudaMemsetAsync(P->status, 0, sizeof(uint32_t), P->st));
  if (st & ST_NONFINITE) return RSVD_ERR_NONFINITE;
  if (st & ST_TIMEOUT) return RSVD_ERR_TIMEOUT;
  if (st & ST_NUMERICAL) return RSVD_ERR_NUMERICAL;
  return RSVD_OK;
}

// Brackets one step: counts its kernel launches and, when the step kind is
// being timed, records a CUDA event pair around it on the plan's stream.
class Step {
 public:
  Step(rsvd_plan_t P, int kind) : P_(P), kind_(kind) {
    if (!(P->prof_mask & (1u << kind))) return;
    auto& v = P->ev[kind];
    int& used = P->ev_used[kind];
    if (used == (int)v.size()) {
      if (used >= 1 << 14) return;  // cap: stop timing rather than grow without bound
      cudaEvent_t a, b;
      if (cudaEventCreate(&a) != cudaSuccess) return;
      if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
      v.emplace_back(a, b);
    }
    end_ = v[used].second;
    cudaEventRecord(v[used].first, P->st);
    ++used;
  }
  ~Step() {
    if (end_) cudaEventRecord(end_, P_->st);
  }
  void launched(int n = 1) { P_->launches[kind_] += n; }

 private:
  rsvd_plan_t P_;
  int kind_;
  cudaEvent_t end_ = nullptr;
};

// ---- the steps --------------------------------------------------------------

// Test matrix (Algorithm 4.1 step 1) into P->omega (n x lp, float32) and, for
// the tensor-core path, its bfloat16 transpose into P->xbf.
rsvd_status_t step_draw(rsvd_plan_t P, bool want_bf16) {
  Step sp(P, RSVD_STEP_DRAW);
  sp.launched();
  if (!P->omega_user && P->opt.test_matrix == RSVD_SRFT) {
    TRY(launch_draw_srft(P->seed, P->n, P->l / 2, P->lp, P->srft_freq, P->omega, P->lp,
                         want_bf16 ? P->xbf : nullptr, tc_ld(P->n), P->st));
  } else if (!P->omega_user) {
    TRY(launch_draw_gaussian(P->seed, 0u, P->n, P->l, P->lp, P->omega, P->lp,
                             want_bf16 ? P->xbf : nullptr, tc_ld(P->n), P->st));
  } else if (want_bf16) {
    TRY(launch_to_bf16_t(P->omega, P->n, P->lp, P->xbf, tc_ld(P->n), 0, 0, P->st));
  }
  return RSVD_OK;
}

// One pass over A (Algorithm 4.4 steps 2, 4, 5; Algorithm 5.1 step 1).
// FP32 path: X is float32 (K x lp); tensor-core path: the operand is P->xbf.
// The result is left as `*splits` partial slabs in P->partial (stride rows x lp).
rsvd_status_t step_pass(rsvd_plan_t P, const void* A, int trans, const float* X, bool split_x,
                        int* splits, int64_t* stride) {
  const int64_t M = trans ? P->n : P->m;
  const int64_t K = trans ? P->m : P->n;
  *stride = M * P->lp;
  Step sp(P, RSVD_STEP_PASS);
  sp.launched();
  if (P->opt.precision == RSVD_PLAIN_FP32) {
    const int s = trans ? P->splits_t : P->splits_n;
    TRY(launch_gemm_f32(trans, M, P->lp, K, static_cast<const float*>(A), P->lda, X, P->lp,
                        P->partial, P->lp, s, *stride, P->st));
    *splits = s;
  } else {
    int s = 1;
    // the residual of A: in the final pass, or in every pass when asked
    const int hilo =
        ((split_x || P->opt.residual_passes) && P->opt.dtype_A == RSVD_BF16X2) ? 1 : 0;
    if (tc_pass(&P->tc, trans, split_x ? 1 : 0, hilo, P->partial, &s, P->st) != 0)
      return RSVD_ERR_CUDA;
    *splits = s;
  }
  return RSVD_OK;
}

// Cholesky-QR rounds on the (summed) partial slabs; the basis ends in `dst`
// (rows x lp).  With `racc`, the triangular factors are multiplied into it.
rsvd_status_t step_orth(rsvd_plan_t P, const float* src, int splits, int64_t stride, int64_t rows,
                        float* dst, float* racc, bool final_basis = true) {
  // A basis that only feeds the next power-iteration pass needs to span the sample, not
  // to be orthonormal to working precision: the shifted round and one plain round leave
  // ||Q^T Q - I|| ~ u kappa(Q_1)^2 with kappa(Q_1) modest after the shift, and the next
  // orthonormalisation starts from the product anyway.  Final bases get every round.
  const int rounds = final_basis ? P->opt.orth_rounds : std::min(P->opt.orth_rounds, 2);
  const int lp = P->lp;
  const int nblk = gram_blocks(rows);
  Step sp(P, RSVD_STEP_ORTH);
  sp.launched(lp <= 128 ? 3 * rounds + 1 : 4 * rounds);
  const float* cur = src;
  int cur_splits = splits;
  if (lp <= 128) {
    // Gram of the sample, then per round: factor, and Q = Y R^-1 fused with the next Gram
    float* yout = (cur_splits > 1) ? P->tmp1 : nullptr;
    TRY(launch_gram_tri(cur, cur_splits, stride, yout, rows, lp, P->gpart, nblk, P->st));
    if (cur_splits > 1) cur = P->tmp1;
    TRY(launch_gram_reduce(P->gpart, nblk, lp, P->g(), P->st));
    for (int r = 0; r < rounds; ++r) {
      const int shifted = (P->opt.orth_rounds >= 3 && r == 0) ? 1 : 0;
      TRY(launch_cholesky(P->g(), P->l, lp, shifted, P->lbuf(), P->rtmp(), P->rinv(), racc,
                          r == 0 ? 1 : 0, P->status, P->st));
      const bool last = (r == rounds - 1);
      float* next = last ? dst : (cur == P->tmp1 ? P->tmp2 : P->tmp1);
      TRY(launch_apply_gram(cur, next, rows, lp, P->rinv(), P->gpart, nblk, last ? 0 : 1, P->st));
      if (!last) TRY(launch_gram_reduce(P->gpart, nblk, lp, P->g(), P->st));
      cur = next;
    }
    return RSVD_OK;
  }
  // Wider bases: on the tensor-core path the Gram partials and Q = Y R^-1 are formed on the
  // tensor cores too (exact three-way bfloat16 splits, six products), else by float32 FMA.  Their float32 accumulation is not IEEE-exact (about
  // 1e-6 of |Y|^T |Y| against 1e-7 for float32 FMA), far below the bfloat16 rounding of A
  // that the path already carries, but not float32-faithful: the plain float32 path keeps
  // the FMA Gram.
  const bool tc_gram = P->opt.precision == RSVD_BF16_TC;
  const int gblk = tc_gram ? gram_tc_grid(rows, nblk) : nblk;
  // per round beyond the Gram, reduce and factorisation: R^-1 by a second kernel for the
  // row-packed factorisation, and the image of R^-1 before the tensor-core apply
  sp.launched(rounds * ((lp / 16 > 10 ? 1 : 0) + (tc_gram ? 1 : 0)));
  for (int r = 0; r < rounds; ++r) {
    float* yout = (cur_splits > 1) ? P->tmp1 : nullptr;
    if (tc_gram)
      TRY(launch_gram_tc(cur, cur_splits, stride, yout, rows, lp, P->gpart, gblk, P->status, P->st));
    else
      TRY(launch_gram_partial(cur, cur_splits, stride, yout, rows, lp, P->gpart, nblk, P->st));
    if (cur_splits > 1) cur = P->tmp1;
    TRY(launch_gram_reduce(P->gpart, gblk, lp, P->g(), P->st));
    const int shifted = (P->opt.orth_rounds >= 3 && r == 0) ? 1 : 0;
    TRY(launch_cholesky(P->g(), P->l, lp, shifted, P->lbuf(), P->rtmp(), P->rinv(), racc,
                        r == 0 ? 1 : 0, P->status, P->st));
    float* next = (r == rounds - 1) ? dst : (cur == P->tmp1 ? P->tmp2 : P->tmp1);
    if (tc_gram)
      TRY(launch_apply_tc(cur, next, rows, lp, P->rinv(), P->rimg, P->status, P->st));
    else
      TRY(launch_gemm_f32(0, rows, lp, lp, cur, lp, P->rinv(), lp, next, lp, 1, 0, P->st));
    cur = next;
    cur_splits = 1;
  }
  return RSVD_OK;
}

// float32 basis (rows x lp) -> transposed bfloat16 operand of the next pass
// (with the lo half when `split`).
rsvd_status_t step_convert(rsvd_plan_t P, const float* x, int64_t rows, int split) {
  Step sp(P, RSVD_STEP_CONVERT);
  sp.launched();
  TRY(launch_to_bf16_t(x, rows, P->lp, P->xbf, tc_ld(rows), split,
                       split ? tc_lo_offset(P->lp) : 0, P->st));
  return RSVD_OK;
}

rsvd_status_t stage_a(rsvd_plan_t P, const void* A) {
  const bool tc = P->opt.precision == RSVD_BF16_TC;
  if (tc)
    TRYS(tc_bind_a(&P->tc, A, P->opt.dtype_A == RSVD_BF16X2) == 0 ? RSVD_OK : RSVD_ERR_CUDA);
  TRYS(step_draw(P, tc));
  int s;
  int64_t stride;
  TRYS(step_pass(P, A, 0, P->omega, false, &s, &stride));
  TRYS(step_orth(P, P->partial, s, stride, P->m, P->qbuf, nullptr, P->q == 0));
  for (int j = 1; j <= P->q; ++j) {
    if (tc) TRYS(step_convert(P, P->qbuf, P->m, 0));
    TRYS(step_pass(P, A, 1, P->qbuf, false, &s, &stride));
    TRYS(step_orth(P, P->partial, s, stride, P->n, P->qtbuf, nullptr, false));
    if (tc) TRYS(step_convert(P, P->qtbuf, P->n, 0));
    TRYS(step_pass(P, A, 0, P->qtbuf, false, &s, &stride));
    TRYS(step_orth(P, P->partial, s, stride, P->m, P->qbuf, nullptr, j == P->q));
  }
  return RSVD_OK;
}

rsvd_status_t stage_b(rsvd_plan_t P, const void* A, float* U, float* S, float* V) {
  const bool tc = P->opt.precision == RSVD_BF16_TC;
  int s;
  int64_t stride;
  if (tc) TRYS(step_convert(P, P->qbuf, P->m, 1));
  TRYS(step_pass(P, A, 1, P->qbuf, true, &s, &stride));      // B^T = A^T Q
  TRYS(step_orth(P, P->partial, s, stride, P->n, P->qtbuf, P->racc()));  // B^T = Q_B R_B
  {
    Step sp(P, RSVD_STEP_SMALL_SVD);
    sp.launched();
    TRY(launch_jacobi_svd(P->racc(), P->lp, 1, P->l, P->lp, P->ut(), P->sig, P->w(), P->lbuf(),
                          P->status, P->status + 1, P->st, P->opt.small_svd));
  }
  Step sp(P, RSVD_STEP_LIFT);
  sp.launched(2);
  TRY(launch_gemm_f32(0, P->m, P->k, P->lp, P->qbuf, P->lp, P->ut(), P->lp, U, P->k, 1, 0, P->st));
  TRY(launch_gemm_f32(0, P->n, P->k, P->lp, P->qtbuf, P->lp, P->w(), P->lp, V, P->k, 1, 0, P->st));
  TRY(cudaMemcpyAsync(S, P->sig, sizeof(float) * P->k, cudaMemcpyDeviceToDevice, P->st));
  return RSVD_OK;
}

rsvd_status_t check_plan(rsvd_plan_t P) {
  if (!P) return RSVD_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return RSVD_ERR_CUDA;
  if (dev != P->device) return RSVD_ERR_INVALID_ARG;
  return RSVD_OK;
}

// Single-pass randomized SVD (Section 5.5): Y = A Omega and Yt = A^T Psi from the
// two sketches alone, Y = Q R and Yt = Qt Rt (Cholesky QR); the bases are cut to the k
// leading left singular vectors Q_k = Q U_R[:, :k], Qt_k = Qt U_Rt[:, :k] (the remedy of
// the section's remark on single-pass error: the systems below become k x l,
// overdetermined), and the reduced k x k matrix B ~ Q_k^T A Qt_k is the minimum-residual
// solution of
//     B X1 = C1,  B^T X2 = C2,   X1 = Qt_k^T Omega, C1 = Q_k^T Y = U_R_k^T R,
//                                X2 = Q_k^T Psi,    C2 = Qt_k^T Yt = U_Rt_k^T Rt,
// i.e. of the Sylvester normal equations (X2 X2^T) B + B (X1 X1^T) = C1 X1^T + X2 C2^T,
// solved in the singular bases of X1 and X2: X_i = U_i S_i W_i^T gives
// B = U2 [(U2^T F U1) ./ (s2_i^2 + s1_j^2)] U1^T, F = C1 X1^T + X2 C2^T.  Then B = Ub Sb Vb^T
// (Jacobi), U = Q (U_R_k Ub), V = Qt (U_Rt_k Vb).  q is ignored; A is read by one pass of
// each kind.
rsvd_status_t stage_single_pass(rsvd_plan_t P, const void* A, float* U, float* S, float* V,
                                float* Qout, int64_t ldq) {
  const bool tc = P->opt.precision == RSVD_BF16_TC;
  const int lp = P->lp, l = P->l;
  const size_t l2 = (size_t)lp * lp;
  if (tc)
    TRYS(tc_bind_a(&P->tc, A, P->opt.dtype_A == RSVD_BF16X2) == 0 ? RSVD_OK : RSVD_ERR_CUDA);
  int s;
  int64_t stride;
  // Y = A Omega, Y = Q R (R accumulated into racc, then kept as C1)
  TRYS(step_draw(P, tc));
  // the cross products below must see the test matrices the bf16 passes multiplied with
  if (tc) TRY(launch_round_bf16(P->omega, P->n, lp, lp, P->st));
  TRYS(step_pass(P, A, 0, P->omega, false, &s, &stride));
  TRYS(step_orth(P, P->partial, s, stride, P->m, P->qbuf, P->racc()));
  TRY(cudaMemcpyAsync(P->sp(2), P->racc(), sizeof(float) * l2, cudaMemcpyDeviceToDevice, P->st));
  if (Qout) TRY(launch_gather(P->qbuf, 1, 0, lp, Qout, ldq, P->m, l, l, P->st));
  // Yt = A^T Psi (Psi: Gaussian, stream 1), Yt = Qt Rt
  {
    Step sp(P, RSVD_STEP_DRAW);
    sp.launched();
    TRY(launch_draw_gaussian(P->seed, 1u, P->m, l, lp, P->psi, lp, tc ? P->xbf : nullptr,
                             tc_ld(P->m), P->st));
    if (tc) TRY(launch_round_bf16(P->psi, P->m, lp, lp, P->st));
  }
  TRYS(step_pass(P, A, 1, P->psi, false, &s, &stride));
  TRYS(step_orth(P, P->partial, s, stride, P->n, P->qtbuf, P->racc()));
  const int k = P->k;
  {
    Step sp(P, RSVD_STEP_SMALL_SVD);
    // (two pairs of Jacobi SVDs run one launch each on the cluster kernel)
    const bool paired = P->opt.small_svd == 2 || (P->opt.small_svd == 0 && l >= 48);
    sp.launched(paired ? 20 : 24);
    // X1 = Qt^T Omega (K = n), X2 = Q^T Psi (K = m): split over row blocks, summed by gather
    const int nblk = std::max(gram_blocks(P->m), gram_blocks(P->n));
    const int s1 = (int)std::min<int64_t>(nblk, std::max<int64_t>(1, cdiv(P->n, 512)));
    TRY(launch_gemm_f32(1, lp, lp, P->n, P->qtbuf, lp, P->omega, lp, P->gpart, lp, s1, l2, P->st));
    TRY(launch_gather(P->gpart, s1, l2, lp, P->sp(0), lp, lp, lp, lp, P->st));
    const int s2 = (int)std::min<int64_t>(nblk, std::max<int64_t>(1, cdiv(P->m, 512)));
    TRY(launch_gemm_f32(1, lp, lp, P->m, P->qbuf, lp, P->psi, lp, P->gpart, lp, s2, l2, P->st));
    TRY(launch_gather(P->gpart, s2, l2, lp, P->sp(1), lp, lp, lp, lp, P->st));
    // the k leading left singular vectors of Y = Q R and Yt = Qt Rt: Q U_R[:, :k], Qt U_Rt[:, :k]
    // (the two SVDs are independent: one launch, one cluster each; the second's discarded W
    // and scratch are the factorisation's buffers, free after the orthonormalisations)
    TRY(launch_jacobi_svd_pair(P->sp(2), P->racc(), lp, 0, l, lp, P->sp(5), P->sp(6), P->sig2,
                               P->sig2 + lp, P->sp(7), P->rtmp(), P->lbuf(), P->rinv(), P->status,
                               P->status + 1, P->st, P->opt.small_svd));
    // the k x l systems: X1 = U_Rt_k^T (Qt^T Omega), C1 = U_R_k^T R, X2 = U_R_k^T (Q^T Psi),
    // C2 = U_Rt_k^T Rt (rows k..l-1 of the padded squares stay zero)
    for (int i : {3, 4, 8, 9}) TRY(cudaMemsetAsync(P->sp(i), 0, sizeof(float) * l2, P->st));
    TRY(launch_small_gemm(k, l, l, 1.f, P->sp(6), lp, 1, P->sp(0), lp, 0, 0.f, P->sp(3), lp, P->st));
    TRY(launch_small_gemm(k, l, l, 1.f, P->sp(5), lp, 1, P->sp(2), lp, 0, 0.f, P->sp(8), lp, P->st));
    TRY(launch_small_gemm(k, l, l, 1.f, P->sp(5), lp, 1, P->sp(1), lp, 0, 0.f, P->sp(4), lp, P->st));
    TRY(launch_small_gemm(k, l, l, 1.f, P->sp(6), lp, 1, P->racc(), lp, 0, 0.f, P->sp(9), lp, P->st));
    // singular bases of X1 (U1 = sp(10), s1) and X2 (U2 = sp(11), s2): k nonzero values each.
    // The one-sided Jacobi runs on X1^T and X2^T: their columns are the k rows of the k x l
    // systems plus l - k zero columns that never rotate, where the l columns of X1 itself
    // would be l vectors in a k-dimensional space, l - k of them rounding noise that no
    // sweep can make orthogonal to the rest.  X^T = Ut S W^T gives X = W S Ut^T: the left
    // singular vectors are the accumulated rotations W.
    TRY(launch_jacobi_svd_pair(P->sp(3), P->sp(4), lp, 1, l, lp, P->sp(7), P->rtmp(), P->sig2,
                               P->sig2 + lp, P->sp(10), P->sp(11), P->lbuf(), P->rinv(), P->status,
                               P->status + 1, P->st, P->opt.small_svd));
    // F = C1 X1^T + X2 C2^T; G = U2^T F U1; H = G ./ (s2^2 + s1^2); B = U2 H U1^T (all k x k)
    TRY(launch_small_gemm(k, k, l, 1.f, P->sp(8), lp, 0, P->sp(3), lp, 1, 0.f, P->sp(12), lp, P->st));
    TRY(launch_small_gemm(k, k, l, 1.f, P->sp(4), lp, 0, P->sp(9), lp, 1, 1.f, P->sp(12), lp, P->st));
    TRY(launch_small_gemm(k, k, k, 1.f, P->sp(11), lp, 1, P->sp(12), lp, 0, 0.f, P->sp(13), lp, P->st));
    TRY(launch_small_gemm(k, k, k, 1.f, P->sp(13), lp, 0, P->sp(10), lp, 0, 0.f, P->sp(12), lp, P->st));
    TRY(launch_sylvester_scale(P->sp(12), k, lp, P->sig2 + lp, P->sig2, P->sp(13), P->st));
    TRY(launch_small_gemm(k, k, k, 1.f, P->sp(11), lp, 0, P->sp(13), lp, 0, 0.f, P->sp(12), lp, P->st));
    TRY(cudaMemsetAsync(P->sq(), 0, sizeof(float) * l2, P->st));
    TRY(launch_small_gemm(k, k, k, 1.f, P->sp(12), lp, 0, P->sp(10), lp, 1, 0.f, P->sq(), lp, P->st));
    // B = Ub Sb Vb^T (k x k), then the lifts' small factors U_R_k Ub and U_Rt_k Vb
    TRY(launch_jacobi_svd(P->sq(), lp, 0, k, lp, P->ut(), P->sig, P->w(), P->lbuf(), P->status,
                          P->status + 1, P->st, P->opt.small_svd));
    TRY(launch_small_gemm(l, k, k, 1.f, P->sp(5), lp, 0, P->ut(), lp, 0, 0.f, P->sp(14), lp, P->st));
    TRY(launch_small_gemm(l, k, k, 1.f, P->sp(6), lp, 0, P->w(), lp, 0, 0.f, P->sp(15), lp, P->st));
  }
  if (!U) return RSVD_OK;
  Step sp(P, RSVD_STEP_LIFT);
  sp.launched(2);
  TRY(launch_gemm_f32(0, P->m, P->k, lp, P->qbuf, lp, P->sp(14), lp, U, P->k, 1, 0, P->st));
  TRY(launch_gemm_f32(0, P->n, P->k, lp, P->qtbuf, lp, P->sp(15), lp, V, P->k, 1, 0, P->st));
  TRY(cudaMemcpyAsync(S, P->sig, sizeof(float) * P->k, cudaMemcpyDeviceToDevice, P->st));
  return RSVD_OK;
}

}  // namespace

extern "C" {

void rsvd_options_default(rsvd_options_t* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->dtype_A = RSVD_F32;
  opt->test_matrix = RSVD_GAUSSIAN;
  opt->precision = RSVD_PLAIN_FP32;
  opt->single_pass = 0;
  opt->recompute = 0;
  opt->orth_rounds = 3;
  opt->lda = 0;
  opt->residual_passes = 0;
  opt->host_f32 = 0;
}

const char* rsvd_status_string(rsvd_status_t s) {
  switch (s) {
    case RSVD_OK: return "success";
    case RSVD_ERR_INVALID_ARG: return "invalid argument";
    case RSVD_ERR_ALLOC: return "allocation failed";
    case RSVD_ERR_CUDA: return "CUDA runtime error";
    case RSVD_ERR_NUMERICAL: return "numerical breakdown";
    case RSVD_ERR_NONFINITE: return "non-finite value in input or intermediate";
    case RSVD_ERR_TIMEOUT: return "bounded device wait expired";
    case RSVD_ERR_UNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

rsvd_status_t rsvd_plan_create(rsvd_plan_t* plan, int64_t m, int64_t n, int32_t k, int32_t p,
                               int32_t q, uint64_t seed, const rsvd_options_t* opt,
                               void* stream) {
  if (!plan) return RSVD_ERR_INVALID_ARG;
  *plan = nullptr;
  rsvd_options_t o;
  if (opt) o = *opt; else rsvd_options_default(&o);
  if (m < 1 || n < 1 || k < 1 || p < 0 || q < 0) return RSVD_ERR_INVALID_ARG;
  const int64_t l = (int64_t)k + p;
  if (l > std::min(m, n) || l > kMaxL) return RSVD_ERR_INVALID_ARG;
  if (o.lda == 0) o.lda = n;
  if (o.lda < n) return RSVD_ERR_INVALID_ARG;
  if (o.orth_rounds != 2 && o.orth_rounds != 3) return RSVD_ERR_INVALID_ARG;
  if (o.dtype_A != RSVD_F32 && o.dtype_A != RSVD_BF16 && o.dtype_A != RSVD_BF16X2)
    return RSVD_ERR_INVALID_ARG;
  if (o.precision == RSVD_PLAIN_FP32 && o.dtype_A != RSVD_F32) return RSVD_ERR_INVALID_ARG;
  if (o.residual_passes != 0 && (o.residual_passes != 1 || o.dtype_A != RSVD_BF16X2))
    return RSVD_ERR_INVALID_ARG;
  if (o.precision == RSVD_BF16_TC && o.dtype_A == RSVD_F32) return RSVD_ERR_INVALID_ARG;
  if (o.precision != RSVD_PLAIN_FP32 && o.precision != RSVD_BF16_TC) return RSVD_ERR_INVALID_ARG;
  if (o.test_matrix != RSVD_GAUSSIAN && o.test_matrix != RSVD_SRFT) return RSVD_ERR_INVALID_ARG;
  // SRFT: l real columns are l / 2 frequencies from {1 .. n/2 - 1} (Section 4.6 for real A)
  if (o.test_matrix == RSVD_SRFT &&
      ((l & 1) || (n & 1) || l / 2 > n / 2 - 1 || n >= ((int64_t)1 << 24)))
    return RSVD_ERR_INVALID_ARG;
  if (o.small_svd < 0 || o.small_svd > 2) return RSVD_ERR_INVALID_ARG;
  if (o.small_svd == 1 && l > 160) return RSVD_ERR_INVALID_ARG;  // one-CTA Jacobi limit
  if (o.precision == RSVD_BF16_TC && (o.lda % 8) != 0) return RSVD_ERR_INVALID_ARG;  // 16-byte rows
  if (o.host_f32 != 0 && (o.host_f32 != 1 || o.precision != RSVD_BF16_TC)) return RSVD_ERR_INVALID_ARG;
  if (o.recompute != 0) return RSVD_ERR_UNSUPPORTED;  // the single-matrix backward keeps no samples

  rsvd_plan_t P = new (std::nothrow) rsvd_plan_s();
  if (!P) return RSVD_ERR_ALLOC;
  P->m = m; P->n = n; P->k = k; P->p = p; P->q = q; P->l = (int)l;
  P->lp = (int)round_up(l, 16);
  P->seed = seed; P->opt = o; P->lda = o.lda;
  P->maxmn = std::max(m, n);
  P->st = static_cast<cudaStream_t>(stream);
  if (cudaGetDevice(&P->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device) !=
          cudaSuccess) {
    cudaGetLastError();
    delete P;
    return RSVD_ERR_CUDA;
  }
  if (prepare_orth() != cudaSuccess || prepare_jacobi() != cudaSuccess ||
      prepare_jacobi_cluster() != cudaSuccess || prepare_gram_tc() != cudaSuccess ||
      prepare_apply_tc() != cudaSuccess) {
    cudaGetLastError();
    delete P;
    return RSVD_ERR_CUDA;
  }
  {
    const char* e = getenv("RSVD_NO_GRAPH");
    P->use_graph = !(e && e[0] && e[0] != '0');
  }
  const int lp = P->lp;
  P->splits_n = choose_splits(m, lp, n, P->num_sms);
  P->splits_t = choose_splits(n, lp, m, P->num_sms);
  int64_t part = std::max((int64_t)P->splits_n * m, (int64_t)P->splits_t * n) * lp;
  if (o.precision == RSVD_BF16_TC) part = std::max(part, tc_partial_elems(m, n, lp, P->num_sms));
  P->partial_elems = part;
  rsvd_status_t s = RSVD_OK;
  const int nblk = std::max(gram_blocks(m), gram_blocks(n));
  if ((s = dalloc(P, &P->omega, (size_t)n * lp)) != RSVD_OK ||
      (s = dalloc(P, &P->qbuf, (size_t)m * lp)) != RSVD_OK ||
      (s = dalloc(P, &P->qtbuf, (size_t)n * lp)) != RSVD_OK ||
      (s = dalloc(P, &P->tmp1, (size_t)P->maxmn * lp)) != RSVD_OK ||
      (s = dalloc(P, &P->tmp2, (size_t)P->maxmn * lp)) != RSVD_OK ||
      (s = dalloc(P, &P->partial, (size_t)part)) != RSVD_OK ||
      (s = dalloc(P, &P->gpart, (size_t)nblk * lp * lp)) != RSVD_OK ||
      (s = dalloc(P, &P->small, (size_t)24 * lp * lp)) != RSVD_OK ||
      (o.single_pass && (s = dalloc(P, &P->psi, (size_t)m * lp)) != RSVD_OK) ||
      (o.single_pass && (s = dalloc(P, &P->sig2, (size_t)2 * lp)) != RSVD_OK) ||
      (s = dalloc(P, &P->sig, (size_t)lp)) != RSVD_OK ||
      (o.test_matrix == RSVD_SRFT && (s = dalloc(P, &P->srft_freq, (size_t)(l / 2))) != RSVD_OK) ||
      (s = dalloc(P, &P->status, 4))) {
    free_plan(P);
    return s;
  }
  if (o.precision == RSVD_BF16_TC && lp > 128 &&
      (s = dalloc(P, &P->rimg, apply_tc_image_bytes(lp))) != RSVD_OK) {
    free_plan(P);
    return s;
  }
  if (o.precision == RSVD_BF16_TC) {
    const size_t xrows = (size_t)tc_lo_offset(lp) + lp;
    if ((s = dalloc(P, &P->xbf, xrows * (size_t)tc_ld(P->maxmn))) != RSVD_OK ||
        cudaMemsetAsync(P->xbf, 0, xrows * (size_t)tc_ld(P->maxmn) * 2, P->st) != cudaSuccess) {
      free_plan(P);
      return s;
    }
    if (tc_plan_init(&P->tc, m, n, o.lda, lp, P->xbf, P->num_sms) != 0) {
      free_plan(P);
      return RSVD_ERR_CUDA;
    }
    P->tc.status = P->status;
  }
  if (o.test_matrix == RSVD_SRFT &&
      launch_srft_select(seed, n, (int)(l / 2), P->srft_freq, P->st) != cudaSuccess) {
    cudaGetLastError();
    free_plan(P);
    return RSVD_ERR_CUDA;
  }
  if (cudaMemsetAsync(P->status, 0, 4 * sizeof(uint32_t), P->st) != cudaSuccess ||
      cudaMemsetAsync(P->small, 0, sizeof(float) * 24 * lp * lp, P->st) != cudaSuccess) {
    free_plan(P);
    return RSVD_ERR_CUDA;
  }
  *plan = P;
  return RSVD_OK;
}

rsvd_status_t rsvd_plan_destroy(rsvd_plan_t P) {
  if (!P) return RSVD_OK;
  cudaStreamSynchronize(P->st);
  free_plan(P);
  return RSVD_OK;
}

rsvd_status_t rsvd_workspace_bytes(rsvd_plan_t P, size_t* bytes) {
  if (!P || !bytes) return RSVD_ERR_INVALID_ARG;
  *bytes = P->ws_bytes;
  return RSVD_OK;
}

rsvd_status_t rsvd_range_finder(rsvd_plan_t P, const void* A, float* Q, int64_t ldq) {
  TRYS(check_plan(P));
  if (!A || !Q || ldq < P->l) return RSVD_ERR_INVALID_ARG;
  if (P->opt.single_pass) return stage_single_pass(P, A, nullptr, nullptr, nullptr, Q, ldq);
  TRYS(stage_a(P, A));
  TRY(launch_gather(P->qbuf, 1, 0, P->lp, Q, ldq, P->m, P->l, P->l, P->st));
  return RSVD_OK;
}

// The kernels of one rsvd_svd call are captured once into a CUDA graph and
// replayed while the plan sees the same A, U, S, V pointers (one launch per call
// instead of about sixty).  Direct launches are used while per-step timing is on,
// on the legacy default stream (which cannot be captured), if capture fails, or
// when the environment sets RSVD_NO_GRAPH=1.
rsvd_status_t run_svd_direct(rsvd_plan_t P, const void* A, float* U, float* S, float* V) {
  if (P->opt.single_pass) return stage_single_pass(P, A, U, S, V, nullptr, 0);
  TRYS(stage_a(P, A));
  TRYS(stage_b(P, A, U, S, V));
  return RSVD_OK;
}

rsvd_status_t rsvd_svd(rsvd_plan_t P, const void* A, float* U, float* S, float* V) {
  TRYS(check_plan(P));
  if (!A || !U || !S || !V) return RSVD_ERR_INVALID_ARG;
  const bool graph_ok = P->use_graph && P->prof_mask == 0 && P->st != nullptr &&
                        P->st != cudaStreamLegacy && P->st != cudaStreamPerThread;
  if (!graph_ok) return run_svd_direct(P, A, U, S, V);
  if (!(P->gexec && P->g_a == A && P->g_u == U && P->g_s == S && P->g_v == V)) {
    if (P->gexec) {
      cudaGraphExecDestroy(P->gexec);
      P->gexec = nullptr;
    }
    int64_t before[RSVD_NUM_STEPS];
    for (int k = 0; k < RSVD_NUM_STEPS; ++k) before[k] = P->launches[k];
    if (cudaStreamBeginCapture(P->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return run_svd_direct(P, A, U, S, V);
    }
    const rsvd_status_t st = run_svd_direct(P, A, U, S, V);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(P->st, &graph);
    if (st != RSVD_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (ce != cudaSuccess || !graph) {
      cudaGetLastError();
      return run_svd_direct(P, A, U, S, V);
    }
    const cudaError_t ie = cudaGraphInstantiate(&P->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      cudaGetLastError();
      P->gexec = nullptr;
      return run_svd_direct(P, A, U, S, V);
    }
    for (int k = 0; k < RSVD_NUM_STEPS; ++k) {
      P->g_launches[k] = P->launches[k] - before[k];
      P->launches[k] = before[k];
    }
    P->g_a = A;
    P->g_u = U;
    P->g_s = S;
    P->g_v = V;
  }
  TRY(cudaGraphLaunch(P->gexec, P->st));
  for (int k = 0; k < RSVD_NUM_STEPS; ++k) P->launches[k] += P->g_launches[k];
  return RSVD_OK;
}

rsvd_status_t rsvd_svd_host(rsvd_plan_t P, const void* A_host, float* U_host, float* S_host,
                            float* V_host) {
  TRYS(check_plan(P));
  if (!A_host || !U_host || !S_host || !V_host) return RSVD_ERR_INVALID_ARG;
  const size_t esz = P->opt.dtype_A == RSVD_F32 ? 4 : 2;
  const bool hilo = P->opt.dtype_A == RSVD_BF16X2;
  const size_t arows = hilo ? 2 * P->m : P->m;
  const size_t abytes = ((size_t)(arows - 1) * P->lda + P->n) * esz;
  const size_t fbytes = ((size_t)(P->m - 1) * P->lda + P->n) * sizeof(float);
  if (!P->a_dev) {
    TRYS(dalloc(P, reinterpret_cast<char**>(&P->a_dev), abytes));
    if (P->opt.host_f32) TRYS(dalloc(P, &P->a_f32, fbytes / sizeof(float)));
    TRYS(dalloc(P, &P->u_dev, (size_t)P->m * P->k));
    TRYS(dalloc(P, &P->s_dev, (size_t)P->k));
    TRYS(dalloc(P, &P->v_dev, (size_t)P->n * P->k));
  }
  if (P->opt.host_f32) {
    // float32 in, the plan's bfloat16 storage (hi, and lo m * lda elements further) out
    TRY(cudaMemcpyAsync(P->a_f32, A_host, fbytes, cudaMemcpyHostToDevice, P->st));
    Step sp(P, RSVD_STEP_CONVERT);
    sp.launched();
    TRY(launch_split_bf16(P->a_f32, P->m, P->n, P->lda, static_cast<__nv_bfloat16*>(P->a_dev),
                          P->lda, hilo ? 1 : 0, P->st));
  } else {
    TRY(cudaMemcpyAsync(P->a_dev, A_host, abytes, cudaMemcpyHostToDevice, P->st));
  }
  TRYS(rsvd_svd(P, P->a_dev, P->u_dev, P->s_dev, P->v_dev));
  TRY(cudaMemcpyAsync(U_host, P->u_dev, sizeof(float) * P->m * P->k, cudaMemcpyDeviceToHost, P->st));
  TRY(cudaMemcpyAsync(S_host, P->s_dev, sizeof(float) * P->k, cudaMemcpyDeviceToHost, P->st));
  TRY(cudaMemcpyAsync(V_host, P->v_dev, sizeof(float) * P->n * P->k, cudaMemcpyDeviceToHost, P->st));
  return take_status(P);
}

rsvd_status_t rsvd_svd_backward(rsvd_plan_t P, const void* A, const float* gU, const float* gS,
                                const float* gV, int32_t add_recon, float* gA) {
  (void)A; (void)gU; (void)gS; (void)gV; (void)add_recon; (void)gA;
  TRYS(check_plan(P));
  return RSVD_ERR_UNSUPPORTED;
}

rsvd_status_t rsvd_get_omega(rsvd_plan_t P, float* Omega) {
  TRYS(check_plan(P));
  if (!Omega) return RSVD_ERR_INVALID_ARG;
  TRYS(step_draw(P, false));
  TRY(launch_gather(P->omega, 1, 0, P->lp, Omega, P->l, P->n, P->l, P->l, P->st));
  return RSVD_OK;
}

rsvd_status_t rsvd_set_omega(rsvd_plan_t P, const float* Omega) {
  TRYS(check_plan(P));
  if (P->gexec) {  // the captured draw no longer matches
    cudaGraphExecDestroy(P->gexec);
    P->gexec = nullptr;
  }
  if (!Omega) {
    P->omega_user = false;
    return RSVD_OK;
  }
  TRY(launch_gather(Omega, 1, 0, P->l, P->omega, P->lp, P->n, P->l, P->lp, P->st));
  P->omega_user = true;
  return RSVD_OK;
}

rsvd_status_t rsvd_sync(rsvd_plan_t P) {
  TRYS(check_plan(P));
  return take_status(P);
}

rsvd_status_t rsvd_diagnostics(rsvd_plan_t P, uint32_t* out, int32_t n) {
  TRYS(check_plan(P));
  if (!out || n < 0) return RSVD_ERR_INVALID_ARG;
  uint32_t w[2] = {0, 0};
  TRY(cudaMemcpyAsync(w, P->status, sizeof(w), cudaMemcpyDeviceToHost, P->st));
  TRY(cudaStreamSynchronize(P->st));
  TRY(cudaMemsetAsync(P->status + 1, 0, sizeof(uint32_t), P->st));
  for (int i = 0; i < n && i < 2; ++i) out[i] = w[i];
  return RSVD_OK;
}

rsvd_status_t rsvd_profile(rsvd_plan_t P, uint32_t mask) {
  TRYS(check_plan(P));
  P->prof_mask = mask;
  for (int k = 0; k < RSVD_NUM_STEPS; ++k) {
    P->ev_used[k] = 0;
    P->launches[k] = 0;
  }
  return RSVD_OK;
}

rsvd_status_t rsvd_profile_read(rsvd_plan_t P, float* ms, int64_t* launches, int32_t nkinds) {
  TRYS(check_plan(P));
  if (nkinds < 0) return RSVD_ERR_INVALID_ARG;
  TRY(cudaStreamSynchronize(P->st));
  for (int k = 0; k < nkinds; ++k) {
    if (k >= RSVD_NUM_STEPS) {
      if (ms) ms[k] = 0.0f;
      if (launches) launches[k] = 0;
      continue;
    }
    if (ms) {
      float tot = 0.0f;
      for (int i = 0; i < P->ev_used[k]; ++i) {
        float t = 0.0f;
        TRY(cudaEventElapsedTime(&t, P->ev[k][i].first, P->ev[k][i].second));
        tot += t;
      }
      ms[k] = tot;
    }
    if (launches) launches[k] = P->launches[k];
  }
  return RSVD_OK;
}

rsvd_status_t rsvd_convert_a(const float* A, int64_t m, int64_t n, int64_t lda, void* out,
                             int64_t ldo, int32_t with_lo, void* stream) {
  if (!A || !out || m < 1 || n < 1 || lda < n || ldo < n) return RSVD_ERR_INVALID_ARG;
  TRY(launch_split_bf16(A, m, n, lda, static_cast<__nv_bfloat16*>(out), ldo, with_lo,
                        static_cast<cudaStream_t>(stream)));
  return RSVD_OK;
}

rsvd_status_t rsvd_draw_gaussian(uint64_t seed, uint32_t stream_id, int64_t rows, int64_t cols,
                                 float* out, int64_t ld, void* stream) {
  if (rows < 0 || cols < 0 || cols > (1 << 30) || (rows > 0 && cols > 0 && !out) || ld < cols)
    return RSVD_ERR_INVALID_ARG;
  TRY(launch_draw_gaussian(seed, stream_id, rows, (int)cols, (int)cols, out, ld, nullptr, 0,
                           static_cast<cudaStream_t>(stream)));
  return RSVD_OK;
}

rsvd_status_t rsvd_sketch(rsvd_plan_t P, const void* A, int32_t transpose, const float* X,
                          float* Y) {
  TRYS(check_plan(P));
  if (!A || !X || !Y) return RSVD_ERR_INVALID_ARG;
  const int64_t kx = transpose ? P->m : P->n;
  const int64_t my = transpose ? P->n : P->m;
  if (P->opt.precision == RSVD_BF16_TC)
    TRYS(tc_bind_a(&P->tc, A, P->opt.dtype_A == RSVD_BF16X2) == 0 ? RSVD_OK : RSVD_ERR_CUDA);
  float* xin = transpose ? P->qbuf : P->omega;  // padded K x lp copy of X
  TRY(launch_gather(X, 1, 0, P->l, xin, P->lp, kx, P->l, P->lp, P->st));
  if (P->opt.precision == RSVD_BF16_TC)
    TRY(launch_to_bf16_t(xin, kx, P->lp, P->xbf, tc_ld(kx), 0, 0, P->st));
  int s;
  int64_t stride;
  TRYS(step_pass(P, A, transpose, xin, false, &s, &stride));
  TRY(launch_gather(P->partial, s, stride, P->lp, Y, P->l, my, P->l, P->l, P->st));
  return RSVD_OK;
}

rsvd_status_t rsvd_orthonormalize(rsvd_plan_t P, int64_t rows, float* Y, float* R) {
  TRYS(check_plan(P));
  if (!Y || rows < P->l || rows > P->maxmn) return RSVD_ERR_INVALID_ARG;
  // the rounds ping-pong through tmp1/tmp2, so the result goes to a basis buffer of `rows` rows
  float* dst = rows <= P->m ? P->qbuf : P->qtbuf;
  TRY(launch_gather(Y, 1, 0, P->l, P->partial, P->lp, rows, P->l, P->lp, P->st));
  TRYS(step_orth(P, P->partial, 1, rows * P->lp, rows, dst, P->racc()));
  TRY(launch_gather(dst, 1, 0, P->lp, Y, P->l, rows, P->l, P->l, P->st));
  if (R) TRY(launch_gather(P->racc(), 1, 0, P->lp, R, P->l, P->l, P->l, P->l, P->st));
  return RSVD_OK;
}

rsvd_status_t rsvd_small_svd(rsvd_plan_t P, const float* X, float* Ut, float* S, float* W) {
  TRYS(check_plan(P));
  if (!X || !Ut || !S || !W) return RSVD_ERR_INVALID_ARG;
  TRY(launch_gather(X, 1, 0, P->l, P->sq(), P->lp, P->l, P->l, P->lp, P->st));
  TRY(launch_jacobi_svd(P->sq(), P->lp, 0, P->l, P->lp, P->ut(), P->sig, P->w(), P->lbuf(),
                        P->status, P->status + 1, P->st, P->opt.small_svd));
  TRY(launch_gather(P->ut(), 1, 0, P->lp, Ut, P->l, P->l, P->l, P->l, P->st));
  TRY(launch_gather(P->w(), 1, 0, P->lp, W, P->l, P->l, P->l, P->l, P->st));
  TRY(cudaMemcpyAsync(S, P->sig, sizeof(float) * P->l, cudaMemcpyDeviceToDevice, P->st));
  return RSVD_OK;
}

}  // extern "C"
