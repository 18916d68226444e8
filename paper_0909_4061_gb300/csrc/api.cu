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
#include <atomic>
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
  int lt = 0, lpp = 0;   // single pass: columns of Psi (l') and their padded width
  int lq = 0;            // the widest padded width, max(lp, lpp): the stride of the small blocks
  uint64_t seed = 0;
  rsvd_options_t opt{};
  cudaStream_t st = nullptr;
  int device = 0, num_sms = kNumSMs;
  int splits_n = 1, splits_t = 1;  // split-K of the passes Y = A X and Y = A^T X (FP32 path)
  int splits_psi = 1;              // split-K of Yt = A^T Psi (FP32 path, single pass)
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
  float* psi = nullptr;      // m x lpp  second test matrix of the single-pass sketch (drawn
                             //          once, at plan creation: it depends on the seed alone)
  float* sig2 = nullptr;     // 2 lp     singular values of X1, X2 (single pass)
  float* sig = nullptr;      // lp
  int* srft_freq = nullptr;  // l / 2 sampled frequencies of the SRFT test matrix
  int* gsrft_perm = nullptr; // the modified SRFT's permutations and rotations (6 n)
  uint32_t* srft_signs = nullptr;  // n bits: the signs d_j of the SRFT (row-transform sketch)
  uint32_t* status = nullptr;
  // backward tape: R^-1 of every Cholesky-QR round of Stage A (always: the factorisation
  // writes it there in place of its scratch block), and in store mode (recompute = 0) the
  // intermediate bases Q_0 .. Q_{q-1}, Qt_1 .. Qt_q
  float* tape_r = nullptr;   // (2q + 1) x 3 x lp x lp: for Y_0 .. Y_q, then Yt_1 .. Yt_q
  float* tape_q = nullptr;   // q x m x lp
  float* tape_qt = nullptr;  // q x n x lp
  bool fwd_ok = false;       // the last call on the plan was rsvd_svd (its state is intact)
  float* bw = nullptr;       // backward workspace (allocated by the first backward call)
  float* ad = nullptr;       // adaptive range finder workspace (its first call)
  float* re = nullptr;       // row ID workspace (its first call): C, candidates, pivots, barrier
  int re_grid = 0;
  int ad_block = 0;
  TcPlan tcb{};              // the tensor-core pass at the adaptive block width
  __nv_bfloat16* xbf = nullptr;  // 2 lp x maxmn: transposed bfloat16 operand of the tensor-core passes
  TcPlan tc{};
  TcPlan tc2{};   // the tensor-core pass at the width of Psi (single pass)
  // rsvd_svd_host staging
  void* a_dev = nullptr;
  float* a_f32 = nullptr;  // float32 staging of A for the host_f32 option
  float *u_dev = nullptr, *s_dev = nullptr, *v_dev = nullptr;
  // the host copy of A in pieces on several streams
  static constexpr int kCopyStreams = 4;
  cudaStream_t cst[kCopyStreams] = {};
  cudaEvent_t cev[kCopyStreams + 1] = {};
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

  // 24 small blocks of lq x lq floats (each holds one padded square of any width <= lq)
  float* g() { return small; }
  float* lbuf() { return small + 1 * (size_t)lq * lq; }
  float* rtmp() { return small + 2 * (size_t)lq * lq; }
  float* rinv() { return small + 3 * (size_t)lq * lq; }
  float* racc() { return small + 4 * (size_t)lq * lq; }
  float* ut() { return small + 5 * (size_t)lq * lq; }
  float* w() { return small + 6 * (size_t)lq * lq; }
  float* sq() { return small + 7 * (size_t)lq * lq; }
  // single pass (Section 5.5): 16 more blocks (see stage_single_pass)
  float* sp(int i) { return small + (size_t)(8 + i) * lq * lq; }
  // where the forward leaves the bases of Stage A: Q_j (j = 0 .. q; Q_q is always qbuf)
  // and Qt_j (j = 1 .. q), and their R factors
  float* basis_q(int j) { return (j < q && tape_q) ? tape_q + (size_t)j * m * lp : qbuf; }
  float* basis_qt(int j) { return tape_qt ? tape_qt + (size_t)(j - 1) * n * lp : qtbuf; }
  float* r_q(int j) { return tape_r ? tape_r + (size_t)j * 3 * lp * lp : nullptr; }
  float* r_qt(int j) { return tape_r ? tape_r + (size_t)(q + j) * 3 * lp * lp : nullptr; }
  int rounds(bool final_basis) const {
    return final_basis ? opt.orth_rounds : std::min(opt.orth_rounds, 2);
  }
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

// Failure injection for tests (rsvd_debug_fail_alloc): the number of device allocations
// still to succeed before one fails, or -1.
std::atomic<int> g_fail_alloc_after{-1};

bool injected_alloc_failure() {
  int v = g_fail_alloc_after.load();
  while (v >= 0) {
    if (g_fail_alloc_after.compare_exchange_weak(v, v - 1)) return v == 0;
  }
  return false;
}

template <class T>
rsvd_status_t dalloc(rsvd_plan_t P, T** ptr, size_t elems) {
  *ptr = nullptr;
  if (elems == 0) elems = 1;
  const size_t bytes = elems * sizeof(T);
  if (injected_alloc_failure()) return RSVD_ERR_ALLOC;
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
  for (cudaStream_t c : P->cst)
    if (c) cudaStreamDestroy(c);
  for (cudaEvent_t e : P->cev)
    if (e) cudaEventDestroy(e);
  void* bufs[] = {P->omega, P->qbuf, P->qtbuf, P->tmp1, P->tmp2, P->partial, P->gpart,
                  P->small, P->sig,  P->status, P->xbf, P->a_dev, P->u_dev, P->s_dev,
                  P->v_dev, P->srft_freq, P->gsrft_perm, P->psi, P->sig2, P->rimg, P->a_f32,
                  P->tape_r, P->tape_q, P->tape_qt, P->bw, P->srft_signs, P->ad, P->re};
  for (void* b : bufs)
    if (b) cudaFree(b);
  tc_plan_destroy(&P->tc);
  tc_plan_destroy(&P->tc2);
  tc_plan_destroy(&P->tcb);
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
  } else if (!P->omega_user && P->opt.test_matrix == RSVD_GSRFT) {
    // the SRFT, then its orthogonal left factor D'' Theta' D' Theta (qtbuf as scratch)
    sp.launched(want_bf16 ? 5 : 4);
    TRY(launch_draw_srft(P->seed, P->n, P->l / 2, P->lp, P->srft_freq, P->omega, P->lp, nullptr, 0,
                         P->st));
    TRY(launch_gsrft_apply(P->seed, P->n, 2 * (P->l / 2), P->lp, P->gsrft_perm, P->omega, P->qtbuf,
                           P->lp, P->st));
    if (want_bf16) TRY(launch_to_bf16_t(P->omega, P->n, P->lp, P->xbf, tc_ld(P->n), 0, 0, P->st));
  } else if (!P->omega_user) {
    TRY(launch_draw_gaussian(P->seed, 0u, P->n, P->l, P->lp, P->omega, P->lp,
                             want_bf16 ? P->xbf : nullptr, tc_ld(P->n), P->st));
  } else if (want_bf16) {
    TRY(launch_to_bf16_t(P->omega, P->n, P->lp, P->xbf, tc_ld(P->n), 0, 0, P->st));
  }
  return RSVD_OK;
}

// The first pass Y = A Omega of an SRFT plan runs as the transform along the rows of A
// (Algorithm 4.5 step 2) when n is a power of two the row-transform kernel takes and the
// test matrix is the plan's own draw.
bool srft_by_fft(rsvd_plan_t P) {
  return P->opt.srft_fft && P->opt.test_matrix == RSVD_SRFT && P->srft_signs != nullptr &&
         !P->omega_user;
}

rsvd_status_t step_srft_fft(rsvd_plan_t P, const void* A, float* out) {
  Step sp(P, RSVD_STEP_PASS);
  sp.launched();
  const bool res = P->opt.residual_passes == 1 || (P->opt.residual_passes == 2 && P->q == 0);
  const int adt = P->opt.dtype_A == RSVD_F32 ? 0 : ((P->opt.dtype_A == RSVD_BF16X2 && res) ? 2 : 1);
  TRY(launch_srft_fft(adt, A, P->lda, P->m, P->n, P->srft_signs, P->srft_freq, P->l / 2, out, P->lp,
                      P->num_sms, P->st));
  return RSVD_OK;
}

// One pass over A (Algorithm 4.4 steps 2, 4, 5; Algorithm 5.1 step 1).
// FP32 path: X is float32 (K x lp); tensor-core path: the operand is P->xbf.
// The result is left as `*splits` partial slabs in P->partial (stride rows x lp).
// final_sample: the pass's output becomes a final basis (the last pass of Stage A), which
// reads the residual of A too when residual_passes = 2.
rsvd_status_t step_pass(rsvd_plan_t P, const void* A, int trans, const float* X, bool split_x,
                        int* splits, int64_t* stride, bool final_sample = false) {
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
    // the residual of A: in the final pass, in every pass (residual_passes = 1) or in the
    // passes whose samples become final bases (residual_passes = 2)
    const bool res = split_x || P->opt.residual_passes == 1 || (P->opt.residual_passes == 2 && final_sample);
    const int hilo = (res && P->opt.dtype_A == RSVD_BF16X2) ? 1 : 0;
    if (tc_pass(&P->tc, trans, split_x ? 1 : 0, hilo, P->partial, &s, P->st) != 0)
      return RSVD_ERR_CUDA;
    *splits = s;
  }
  return RSVD_OK;
}

// Yt = A^T Psi at the width of Psi (single pass): the second tensor-core plan or the
// float32 GEMM with lpp columns; the result stays in P->partial as `*splits` slabs.
rsvd_status_t step_pass_psi(rsvd_plan_t P, const void* A, int* splits, int64_t* stride) {
  *stride = P->n * P->lpp;
  Step sp(P, RSVD_STEP_PASS);
  sp.launched();
  if (P->opt.precision == RSVD_PLAIN_FP32) {
    TRY(launch_gemm_f32(1, P->n, P->lpp, P->m, static_cast<const float*>(A), P->lda, P->psi, P->lpp,
                        P->partial, P->lpp, P->splits_psi, *stride, P->st));
    *splits = P->splits_psi;
  } else {
    int s = 1;
    const int hilo = (P->opt.residual_passes && P->opt.dtype_A == RSVD_BF16X2) ? 1 : 0;
    if (tc_pass(&P->tc2, 1, 0, hilo, P->partial, &s, P->st) != 0) return RSVD_ERR_CUDA;
    *splits = s;
  }
  return RSVD_OK;
}

// Cholesky-QR rounds on the (summed) partial slabs; the basis ends in `dst`
// (rows x lp).  With `racc`, the triangular factors are multiplied into it.
rsvd_status_t step_orth(rsvd_plan_t P, const float* src, int splits, int64_t stride, int64_t rows,
                        float* dst, float* racc, bool final_basis = true, int width = 0,
                        float* rinv_tape = nullptr) {
  // A basis that only feeds the next power-iteration pass needs to span the sample, not
  // to be orthonormal to working precision: the shifted round and one plain round leave
  // ||Q^T Q - I|| ~ u kappa(Q_1)^2 with kappa(Q_1) modest after the shift, and the next
  // orthonormalisation starts from the product anyway.  Final bases get every round.
  // width: the columns of the sample (0: l; the single pass also orthonormalises the l'
  // columns of A^T Psi).
  // rinv_tape: R^-1 of round r goes to rinv_tape + r lp^2 (the backward's tape) instead of
  // the scratch block
  const int rounds = P->rounds(final_basis);
  const int wl = width ? width : P->l;
  const int lp = (int)round_up(wl, 16);
  auto ri = [&](int r) { return rinv_tape ? rinv_tape + (size_t)r * lp * lp : P->rinv(); };
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
      TRY(launch_cholesky(P->g(), wl, lp, shifted, P->lbuf(), P->rtmp(), ri(r), racc,
                          r == 0 ? 1 : 0, P->status, P->st));
      const bool last = (r == rounds - 1);
      float* next = last ? dst : (cur == P->tmp1 ? P->tmp2 : P->tmp1);
      TRY(launch_apply_gram(cur, next, rows, lp, ri(r), P->gpart, nblk, last ? 0 : 1, P->st));
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
    TRY(launch_cholesky(P->g(), wl, lp, shifted, P->lbuf(), P->rtmp(), ri(r), racc,
                        r == 0 ? 1 : 0, P->status, P->st));
    float* next = (r == rounds - 1) ? dst : (cur == P->tmp1 ? P->tmp2 : P->tmp1);
    if (tc_gram)
      TRY(launch_apply_tc(cur, next, rows, lp, ri(r), P->rimg, P->status, P->st));
    else
      TRY(launch_gemm_f32(0, rows, lp, lp, cur, lp, ri(r), lp, next, lp, 1, 0, P->st));
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
  int s;
  int64_t stride;
  // Y_0 = A Omega: the SRFT by its transform along the rows (no n x l matrix), else a pass
  // with the drawn test matrix
  if (srft_by_fft(P)) {
    TRYS(step_srft_fft(P, A, P->partial));
    s = 1;
    stride = P->m * P->lp;
  } else {
    TRYS(step_draw(P, tc));
    TRYS(step_pass(P, A, 0, P->omega, false, &s, &stride, P->q == 0));
  }
  // the bases go where the backward finds them (the tape in store mode), with their R factors
  TRYS(step_orth(P, P->partial, s, stride, P->m, P->basis_q(0), nullptr, P->q == 0, 0, P->r_q(0)));
  for (int j = 1; j <= P->q; ++j) {
    if (tc) TRYS(step_convert(P, P->basis_q(j - 1), P->m, 0));
    TRYS(step_pass(P, A, 1, P->basis_q(j - 1), false, &s, &stride));
    TRYS(step_orth(P, P->partial, s, stride, P->n, P->basis_qt(j), nullptr, false, 0, P->r_qt(j)));
    if (tc) TRYS(step_convert(P, P->basis_qt(j), P->n, 0));
    TRYS(step_pass(P, A, 0, P->basis_qt(j), false, &s, &stride, j == P->q));
    TRYS(step_orth(P, P->partial, s, stride, P->m, P->basis_q(j), nullptr, j == P->q, 0, P->r_q(j)));
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

// Single-pass randomized SVD (Section 5.5): Y = A Omega (n x l) and Yt = A^T Psi (Psi m x l')
// from the two sketches alone, Y = Q R and Yt = Qt Rt (Cholesky QR); the bases are cut to
// the k leading left singular vectors Q_k = Q U_R[:, :k], Qt_k = Qt U_Rt[:, :k] (the remedy
// of the section's remark on single-pass error: the systems below become k x l and
// k x l', overdetermined), and the reduced k x k matrix B ~ Q_k^T A Qt_k is the
// minimum-residual solution of
//     B X1 = C1,  B^T X2 = C2,   X1 = Qt_k^T Omega (k x l),  C1 = Q_k^T Y = U_R_k^T R,
//                                X2 = Q_k^T Psi (k x l'),    C2 = Qt_k^T Yt = U_Rt_k^T Rt,
// i.e. of the Sylvester normal equations (X2 X2^T) B + B (X1 X1^T) = C1 X1^T + X2 C2^T,
// solved in the eigenbases of the two k x k Gram matrices: X1 X1^T = U1 L1 U1^T,
// X2 X2^T = U2 L2 U2^T give B = U2 [(U2^T F U1) ./ (L2_i + L1_j)] U1^T, F = C1 X1^T + X2 C2^T
// (the eigendecompositions come from the one-sided Jacobi SVD of the symmetric positive
// semidefinite Grams).  Then B = Ub Sb Vb^T (Jacobi), U = Q (U_R_k Ub), V = Qt (U_Rt_k Vb).
// q is ignored; A is read by one pass of each kind.
// Small blocks: R (lp, ld lp), Rt (lpp, ld lpp), the k x k matrices with ld kp = k rounded
// up to 16.
rsvd_status_t stage_single_pass(rsvd_plan_t P, const void* A, float* U, float* S, float* V,
                                float* Qout, int64_t ldq) {
  const bool tc = P->opt.precision == RSVD_BF16_TC;
  const int lp = P->lp, l = P->l, lpp = P->lpp, lt = P->lt, lq = P->lq, k = P->k;
  const int kp = (int)round_up(k, 16);
  if (tc) {
    const int lo = P->opt.dtype_A == RSVD_BF16X2;
    if (tc_bind_a(&P->tc, A, lo) != 0 || tc_bind_a(&P->tc2, A, lo) != 0) return RSVD_ERR_CUDA;
  }
  int s;
  int64_t stride;
  // Y = A Omega, Y = Q R (R kept in sp(2))
  TRYS(step_draw(P, tc));
  // the cross products below must see the test matrices the bf16 passes multiplied with
  if (tc) TRY(launch_round_bf16(P->omega, P->n, lp, lp, P->st));
  TRYS(step_pass(P, A, 0, P->omega, false, &s, &stride, true));
  TRYS(step_orth(P, P->partial, s, stride, P->m, P->qbuf, P->sp(2)));
  if (Qout) TRY(launch_gather(P->qbuf, 1, 0, lp, Qout, ldq, P->m, l, l, P->st));
  // Yt = A^T Psi (Psi: Gaussian, stream 1, l' columns), Yt = Qt Rt (Rt in racc, ld lpp)
  // Psi (drawn at plan creation, float32 holding the bfloat16 values the tensor-core pass
  // multiplies with): its transposed bfloat16 operand, which other passes overwrite
  if (tc) {
    Step sp(P, RSVD_STEP_CONVERT);
    sp.launched();
    TRY(launch_to_bf16_t(P->psi, P->m, lpp, P->xbf, tc_ld(P->m), 0, 0, P->st));
  }
  TRYS(step_pass_psi(P, A, &s, &stride));
  TRYS(step_orth(P, P->partial, s, stride, P->n, P->qtbuf, P->racc(), true, lt));
  {
    Step sp(P, RSVD_STEP_SMALL_SVD);
    sp.launched(23);
    // X1 = Qt^T Omega (lpp x lp, K = n), X2 = Q^T Psi (lp x lpp, K = m): row blocks, summed
    const int nblk = std::max(gram_blocks(P->m), gram_blocks(P->n));
    const int s1 = (int)std::min<int64_t>(nblk, std::max<int64_t>(1, cdiv(P->n, 512)));
    const int64_t l12 = (int64_t)lpp * lp;
    TRY(launch_gemm_f32(1, lpp, lp, P->n, P->qtbuf, lpp, P->omega, lp, P->gpart, lp, s1, l12, P->st));
    TRY(launch_gather(P->gpart, s1, l12, lp, P->sp(0), lp, lpp, lp, lp, P->st));
    const int s2 = (int)std::min<int64_t>(nblk, std::max<int64_t>(1, cdiv(P->m, 512)));
    TRY(launch_gemm_f32(1, lp, lpp, P->m, P->qbuf, lp, P->psi, lpp, P->gpart, lpp, s2, l12, P->st));
    TRY(launch_gather(P->gpart, s2, l12, lpp, P->sp(1), lpp, lp, lpp, lpp, P->st));
    // the left singular vectors of R and of Rt: U_R (sp(5), ld lp), U_Rt (sp(6), ld lpp)
    TRY(launch_jacobi_svd(P->sp(2), lp, 0, l, lp, P->sp(5), P->sig2, P->sp(7), P->lbuf(), P->status,
                          P->status + 1, P->st, P->opt.small_svd == 1 && l > 160 ? 0 : P->opt.small_svd));
    TRY(launch_jacobi_svd(P->racc(), lpp, 0, lt, lpp, P->sp(6), P->sig2 + lq, P->rtmp(), P->lbuf(),
                          P->status, P->status + 1, P->st,
                          P->opt.small_svd == 1 && lt > 160 ? 0 : P->opt.small_svd));
    // the k x l and k x l' systems (sp(3) X1_k, sp(8) C1: ld lp; sp(4) X2_k, sp(9) C2: ld lpp)
    for (int i : {3, 4, 8, 9}) TRY(cudaMemsetAsync(P->sp(i), 0, sizeof(float) * lq * lq, P->st));
    TRY(launch_small_gemm(k, l, lt, 1.f, P->sp(6), lpp, 1, P->sp(0), lp, 0, 0.f, P->sp(3), lp, P->st));
    TRY(launch_small_gemm(k, l, l, 1.f, P->sp(5), lp, 1, P->sp(2), lp, 0, 0.f, P->sp(8), lp, P->st));
    TRY(launch_small_gemm(k, lt, l, 1.f, P->sp(5), lp, 1, P->sp(1), lpp, 0, 0.f, P->sp(4), lpp, P->st));
    TRY(launch_small_gemm(k, lt, lt, 1.f, P->sp(6), lpp, 1, P->racc(), lpp, 0, 0.f, P->sp(9), lpp, P->st));
    // the normal-equation matrices G1 = X1_k X1_k^T, G2 = X2_k X2_k^T (k x k, ld kp) and their
    // eigenbases (U1 in sp(10), U2 in sp(11); eigenvalues in sig2 and sig2 + lq)
    for (int i : {12, 13}) TRY(cudaMemsetAsync(P->sp(i), 0, sizeof(float) * lq * lq, P->st));
    TRY(launch_small_gemm(k, k, l, 1.f, P->sp(3), lp, 0, P->sp(3), lp, 1, 0.f, P->sp(12), kp, P->st));
    TRY(launch_small_gemm(k, k, lt, 1.f, P->sp(4), lpp, 0, P->sp(4), lpp, 1, 0.f, P->sp(13), kp, P->st));
    TRY(launch_jacobi_svd_pair(P->sp(12), P->sp(13), kp, 0, k, kp, P->sp(10), P->sp(11), P->sig2,
                               P->sig2 + lq, P->sp(7), P->rtmp(), P->lbuf(), P->rinv(), P->status,
                               P->status + 1, P->st, P->opt.small_svd));
    // F = C1 X1_k^T + X2_k C2^T; G = U2^T F U1; H = G ./ (L2_i + L1_j); B = U2 H U1^T (k x k)
    TRY(launch_small_gemm(k, k, l, 1.f, P->sp(8), lp, 0, P->sp(3), lp, 1, 0.f, P->sp(12), kp, P->st));
    TRY(launch_small_gemm(k, k, lt, 1.f, P->sp(4), lpp, 0, P->sp(9), lpp, 1, 1.f, P->sp(12), kp, P->st));
    TRY(launch_small_gemm(k, k, k, 1.f, P->sp(11), kp, 1, P->sp(12), kp, 0, 0.f, P->sp(13), kp, P->st));
    TRY(launch_small_gemm(k, k, k, 1.f, P->sp(13), kp, 0, P->sp(10), kp, 0, 0.f, P->sp(12), kp, P->st));
    TRY(launch_sylvester_scale(P->sp(12), k, kp, P->sig2 + lq, P->sig2, 1, P->sp(13), P->st));
    TRY(launch_small_gemm(k, k, k, 1.f, P->sp(11), kp, 0, P->sp(13), kp, 0, 0.f, P->sp(12), kp, P->st));
    TRY(cudaMemsetAsync(P->sq(), 0, sizeof(float) * lq * lq, P->st));
    TRY(launch_small_gemm(k, k, k, 1.f, P->sp(12), kp, 0, P->sp(10), kp, 1, 0.f, P->sq(), kp, P->st));
    // B = Ub Sb Vb^T (k x k), then the lifts' small factors U_R_k Ub (l x k) and U_Rt_k Vb
    // (l' x k), rows beyond l and l' zero (sp(14), sp(15), ld kp)
    TRY(launch_jacobi_svd(P->sq(), kp, 0, k, kp, P->ut(), P->sig, P->w(), P->lbuf(), P->status,
                          P->status + 1, P->st, P->opt.small_svd));
    for (int i : {14, 15}) TRY(cudaMemsetAsync(P->sp(i), 0, sizeof(float) * lq * lq, P->st));
    TRY(launch_small_gemm(l, k, k, 1.f, P->sp(5), lp, 0, P->ut(), kp, 0, 0.f, P->sp(14), kp, P->st));
    TRY(launch_small_gemm(lt, k, k, 1.f, P->sp(6), lpp, 0, P->w(), kp, 0, 0.f, P->sp(15), kp, P->st));
  }
  if (!U) return RSVD_OK;
  Step sp(P, RSVD_STEP_LIFT);
  sp.launched(2);
  TRY(launch_gemm_f32(0, P->m, P->k, lp, P->qbuf, lp, P->sp(14), kp, U, P->k, 1, 0, P->st));
  TRY(launch_gemm_f32(0, P->n, P->k, lpp, P->qtbuf, lpp, P->sp(15), kp, V, P->k, 1, 0, P->st));
  TRY(cudaMemcpyAsync(S, P->sig, sizeof(float) * P->k, cudaMemcpyDeviceToDevice, P->st));
  return RSVD_OK;
}

// ---- adaptive range finder (Algorithm 4.2, blocked; the fixed-precision problem) ----------
//
// The sample stream is the n x (l_p + b) Gaussian matrix of Philox stream 3 (block t is its
// columns (t - 1) b .. t b - 1).  Per block: the posterior estimate max_i ||(I - Q Q^T) A w_i||
// over the block's samples (read by the host); if it is above eps / (10 sqrt(2/pi)) (4.3),
// the block is reprojected, orthonormalised (Cholesky QR), reprojected once normalised and
// orthonormalised again, and appended to Q; then the next block is sampled and projected.
constexpr uint32_t kStreamAdaptive = 3u;

struct Ad {
  float *om, *y, *qb, *c, *g;
};

void ad_layout(rsvd_plan_t P, int b, Ad* w, float* base) {
  const size_t n = P->n, m = P->m, lp = P->lp;
  size_t off = 0;
  auto take = [&](float** p, size_t elems) {
    *p = base ? base + off : nullptr;
    off += (elems + 63) & ~size_t(63);
  };
  take(&w->om, n * (lp + b));
  take(&w->y, m * b);
  take(&w->qb, m * b);
  take(&w->c, lp * (size_t)b);
  take(&w->g, (size_t)b * b);
  (void)off;
}

size_t ad_elems(rsvd_plan_t P, int b) {
  const size_t n = P->n, m = P->m, lp = P->lp;
  auto r = [](size_t e) { return (e + 63) & ~size_t(63); };
  return r(n * (lp + b)) + 2 * r(m * b) + r(lp * (size_t)b) + r((size_t)b * b);
}

// out (m x b) = A X for a float32 X (n x b, leading dimension b) at the block width
rsvd_status_t ad_pass(rsvd_plan_t P, const void* A, const float* X, int b, float* out) {
  Step sp(P, RSVD_STEP_PASS);
  int s = 1;
  const int64_t stride = P->m * b;
  if (P->opt.precision == RSVD_PLAIN_FP32) {
    sp.launched(2);
    s = choose_splits(P->m, b, P->n, P->num_sms);
    TRY(launch_gemm_f32(0, P->m, b, P->n, static_cast<const float*>(A), P->lda, X, b, P->partial, b, s,
                        stride, P->st));
  } else {
    sp.launched(3);
    TRY(launch_to_bf16_t(X, P->n, b, P->xbf, tc_ld(P->n), 0, 0, P->st));
    const int hilo = (P->opt.residual_passes && P->opt.dtype_A == RSVD_BF16X2) ? 1 : 0;
    if (tc_pass(&P->tcb, 0, 0, hilo, P->partial, &s, P->st) != 0) return RSVD_ERR_CUDA;
  }
  TRY(launch_gather(P->partial, s, stride, b, out, b, P->m, b, b, P->st));
  return RSVD_OK;
}

// y <- (I - Q Q^T) y for the first j columns of Q (ld lp) and y (m x b)
rsvd_status_t ad_project(rsvd_plan_t P, const Ad& w, int j, int b, float* y) {
  if (j == 0) return RSVD_OK;
  const int lp = P->lp;
  const int nblk = std::max(gram_blocks(P->m), gram_blocks(P->n));
  const int s = (int)std::min<int64_t>(nblk, std::max<int64_t>(1, cdiv(P->m, 512)));
  const int64_t stride = (int64_t)j * b;
  TRY(launch_gemm_f32(1, j, b, P->m, P->qbuf, lp, y, b, P->gpart, b, s, stride, P->st));
  TRY(launch_gather(P->gpart, s, stride, b, w.c, b, j, b, b, P->st));
  TRY(launch_small_gemm((int)P->m, b, j, -1.0f, P->qbuf, lp, 0, w.c, b, 0, 1.0f, y, b, P->st));
  return RSVD_OK;
}

// the largest column norm of y (m x b): the diagonal of y^T y, summed in row blocks
rsvd_status_t ad_estimate(rsvd_plan_t P, const Ad& w, int b, const float* y, float* est) {
  const int nblk = std::max(gram_blocks(P->m), gram_blocks(P->n));
  const int s = (int)std::min<int64_t>(nblk, std::max<int64_t>(1, cdiv(P->m, 512)));
  const int64_t stride = (int64_t)b * b;
  TRY(launch_gemm_f32(1, b, b, P->m, y, b, y, b, P->gpart, b, s, stride, P->st));
  TRY(launch_gather(P->gpart, s, stride, b, w.g, b, b, b, b, P->st));
  std::vector<float> g((size_t)b * b);
  TRY(cudaMemcpyAsync(g.data(), w.g, sizeof(float) * b * b, cudaMemcpyDeviceToHost, P->st));
  TRY(cudaStreamSynchronize(P->st));
  float mx = 0.0f;
  for (int i = 0; i < b; ++i) mx = std::max(mx, g[(size_t)i * b + i]);
  *est = sqrtf(std::max(mx, 0.0f));
  return RSVD_OK;
}

rsvd_status_t run_adaptive(rsvd_plan_t P, const void* A, float eps, int b, float* Q, int64_t ldq,
                           int32_t* rank, float* estimate) {
  const bool tc = P->opt.precision == RSVD_BF16_TC;
  const int lp = P->lp, cap = P->l;
  if (!P->ad || P->ad_block != b) {
    if (P->ad) {
      cudaFree(P->ad);
      P->ad = nullptr;
    }
    tc_plan_destroy(&P->tcb);
    TRYS(dalloc(P, &P->ad, ad_elems(P, b)));
    P->ad_block = b;
    if (tc) {
      if (tc_plan_init(&P->tcb, P->m, P->n, P->lda, b, P->xbf, P->num_sms) != 0) return RSVD_ERR_CUDA;
      P->tcb.status = P->status;
    }
  }
  Ad w;
  ad_layout(P, b, &w, P->ad);
  if (tc && tc_bind_a(&P->tcb, A, P->opt.dtype_A == RSVD_BF16X2) != 0) return RSVD_ERR_CUDA;
  {
    Step sp(P, RSVD_STEP_DRAW);
    sp.launched();
    TRY(launch_draw_gaussian(P->seed, kStreamAdaptive, P->n, lp + b, lp + b, w.om, lp + b, nullptr, 0,
                             P->st));
  }
  // block t of the sample stream as an n x b matrix (leading dimension b)
  auto sample = [&](int t, float* out) -> rsvd_status_t {
    TRY(launch_gather(w.om + (size_t)t * b, 1, 0, lp + b, P->qtbuf, b, P->n, b, b, P->st));
    return ad_pass(P, A, P->qtbuf, b, out);
  };
  const float thresh = eps / (10.0f * sqrtf(2.0f / 3.14159265358979f));
  int j = 0, t = 0;
  TRYS(sample(t++, w.y));
  float est = 0.0f;
  for (;;) {
    TRYS(ad_estimate(P, w, b, w.y, &est));
    if (!(est > thresh) || j + b > cap) break;
    // steps 7-8 for the block: reproject, orthonormalise, reproject, orthonormalise
    TRYS(ad_project(P, w, j, b, w.y));
    TRYS(step_orth(P, w.y, 1, P->m * b, P->m, w.qb, nullptr, true, b));
    TRYS(ad_project(P, w, j, b, w.qb));
    TRYS(step_orth(P, w.qb, 1, P->m * b, P->m, w.y, nullptr, true, b));
    TRY(launch_gather(w.y, 1, 0, b, P->qbuf + j, lp, P->m, b, b, P->st));
    j += b;
    // steps 10-11: the next block of samples, projected
    TRYS(sample(t++, w.y));
    TRYS(ad_project(P, w, j, b, w.y));
  }
  if (j > 0) TRY(launch_gather(P->qbuf, 1, 0, lp, Q, ldq, P->m, j, j, P->st));
  *rank = j;
  if (estimate) *estimate = est;
  return RSVD_OK;
}

// ---- backward (reverse mode through Algorithm 4.4 + Algorithm 5.1, Omega fixed) ----------
//
// Forward map: Y_0 = A Omega = Q_0 R_0; Yt_j = A^T Q_{j-1} = Qt_j Rt_j, Y_j = A Qt_j = Q_j R_j
// (j = 1 .. q); B = Q_q^T A = Ut S V_B^T (the thin SVD, computed as B^T = Q_B R_B and
// R_B^T = Ut S W^T, V_B = Q_B W); U = Q_q Ut_k, S = S_k, V = V_B_k.
// Given the cotangents gU, gS, gV (and the loss ||A - U S V^T||_F^2 + sum S when add_recon):
//   SVD of B:   J = Ut^T (Q^T gU), K = V_B^T gV, M = F o (J - J^T) S + S F o (K - K^T) + diag gS,
//               gB^T = Z Ut^T with Z = V_B (M^T - K S^-1) + gV S^-1   (F_ij = 1 / (s_j^2 - s_i^2))
//   B = Q^T A:  gA += (Q Ut) Z^T,  gQ = (gU | 0) Ut^T + (A Z) Ut^T
//   Y = Q R:    gY = (gQ + Q copyltu(-gQ^T Q)) R^-T          (R itself unused downstream)
//   Y = A X:    gA += gY X^T,  gX = A^T gY;   Y = A^T X likewise
// and with add_recon the reconstruction term adds 2 A - 2 U S V^T to gA and
// 2 S^2 U - 2 (A V) S to gU, 1 to gS (U^T A V = S and A^T U = V S for the exact SVD of B).
// gA = alpha A + L R^T is formed by one tiled product over the stacked factors (store
// mode), or pair by pair (recompute mode, which keeps no stack and recomputes the
// intermediate bases of Stage A from A).
struct Bw {
  // m side (rows m x lp), n side (rows n x lp), small (lp x lp)
  float *gq, *tm, *ufull, *pm;
  float *vb, *z, *tn, *gqt;
  float *J, *K, *M2, *C, *N, *rinv, *utc, *wc, *t1, *gst;
  float *wq0, *wq1, *wqt;      // recompute mode: Q_{j-1} / Q_j (ping-pong) and Qt_j
  float *lf, *rf;              // store mode: the stacked factors (m x kr, n x kr)
  int kr;
};

size_t bw_layout(rsvd_plan_t P, Bw* b, float* base) {
  const size_t m = P->m, n = P->n, lp = P->lp, l2 = lp * lp;
  const bool store = P->opt.recompute == 0;
  const int blocks = 2 * P->q + 3;   // (recon) + (U_full, Z) + 2 per power step + (gY_0, Omega)
  b->kr = blocks * (int)lp;
  size_t off = 0;
  auto take = [&](float** p, size_t elems) {
    *p = base ? base + off : nullptr;
    off += (elems + 63) & ~size_t(63);
  };
  take(&b->gq, m * lp); take(&b->tm, m * lp); take(&b->ufull, m * lp); take(&b->pm, m * lp);
  take(&b->vb, n * lp); take(&b->z, n * lp); take(&b->tn, n * lp); take(&b->gqt, n * lp);
  for (float** p : {&b->J, &b->K, &b->M2, &b->C, &b->N, &b->rinv, &b->utc, &b->wc, &b->t1})
    take(p, l2);
  take(&b->gst, lp);
  b->wq0 = b->wq1 = b->wqt = b->lf = b->rf = nullptr;
  if (store) {
    take(&b->lf, m * (size_t)b->kr);
    take(&b->rf, n * (size_t)b->kr);
  } else {
    take(&b->wq0, m * lp); take(&b->wq1, m * lp); take(&b->wqt, n * lp);
  }
  return off;
}

// out (rows_out x lp) = A X or A^T X for a float32 X (rows_in x lp): one pass with the plan's
// precision; on the tensor cores X goes in as a bfloat16 hi + lo pair (and A as hi + lo
// when stored so), so the product carries about 16 bits of the operand.
rsvd_status_t bw_pass(rsvd_plan_t P, const void* A, int trans, const float* X, float* out) {
  const int64_t rows_in = trans ? P->m : P->n, rows_out = trans ? P->n : P->m;
  const int lp = P->lp;
  int s = 1;
  int64_t stride = rows_out * lp;
  Step sp(P, RSVD_STEP_PASS);
  sp.launched(P->opt.precision == RSVD_BF16_TC ? 3 : 2);
  if (P->opt.precision == RSVD_PLAIN_FP32) {
    s = trans ? P->splits_t : P->splits_n;
    TRY(launch_gemm_f32(trans, rows_out, lp, rows_in, static_cast<const float*>(A), P->lda, X, lp,
                        P->partial, lp, s, stride, P->st));
  } else {
    TRY(launch_to_bf16_t(X, rows_in, lp, P->xbf, tc_ld(rows_in), 1, tc_lo_offset(lp), P->st));
    const int hilo = P->opt.dtype_A == RSVD_BF16X2 ? 1 : 0;
    if (tc_pass(&P->tc, trans, 1, hilo, P->partial, &s, P->st) != 0) return RSVD_ERR_CUDA;
  }
  TRY(launch_gather(P->partial, s, stride, lp, out, lp, rows_out, lp, lp, P->st));
  return RSVD_OK;
}

// out (lp x ncols, ld lp, zero-padded to lp columns) = X^T Y for X (rows x lp), Y (rows x
// ncols, ld ldy): row blocks as split-K partials, summed in a fixed order.
rsvd_status_t bw_tn(rsvd_plan_t P, int64_t rows, const float* X, const float* Y, int ldy, int ncols,
                    float* out) {
  const int lp = P->lp;
  const int nblk = std::max(gram_blocks(P->m), gram_blocks(P->n));
  const int s = (int)std::min<int64_t>(nblk, std::max<int64_t>(1, cdiv(rows, 512)));
  const int64_t l2 = (int64_t)lp * lp;
  TRY(launch_gemm_f32(1, lp, ncols, rows, X, lp, Y, ldy, P->gpart, lp, s, l2, P->st));
  TRY(launch_gather(P->gpart, s, l2, lp, out, lp, lp, ncols, lp, P->st));
  return RSVD_OK;
}

// gY = (gQ + Q copyltu(-gQ^T Q)) R^-T for Y = Q R (rows x lp), R = R_r ... R_1 the product
// of the Cholesky-QR rounds, so R^-1 = R_1^-1 ... R_r^-1 from the rounds' inverses on the tape
rsvd_status_t bw_qr(rsvd_plan_t P, Bw& b, int64_t rows, const float* Q, const float* gQ,
                    const float* rinv_rounds, int rounds, float* T, float* gY) {
  const int lp = P->lp;
  const size_t l2 = (size_t)lp * lp;
  TRYS(bw_tn(P, rows, gQ, Q, lp, lp, b.C));
  TRY(launch_copyltu_neg(b.C, lp, b.N, P->st));
  TRY(launch_gather(gQ, 1, 0, lp, T, lp, rows, lp, lp, P->st));
  TRY(launch_small_gemm((int)rows, lp, lp, 1.0f, Q, lp, 0, b.N, lp, 0, 1.0f, T, lp, P->st));
  const float* rinv = rinv_rounds;
  if (rounds > 1) {
    float* acc[2] = {b.rinv, b.t1};
    TRY(launch_small_gemm(lp, lp, lp, 1.0f, rinv_rounds, lp, 0, rinv_rounds + l2, lp, 0, 0.0f, acc[0],
                          lp, P->st));
    int cur = 0;
    for (int r = 2; r < rounds; ++r, cur ^= 1)
      TRY(launch_small_gemm(lp, lp, lp, 1.0f, acc[cur], lp, 0, rinv_rounds + r * l2, lp, 0, 0.0f,
                            acc[cur ^ 1], lp, P->st));
    rinv = acc[cur];
  }
  TRY(launch_small_gemm((int)rows, lp, lp, 1.0f, T, lp, 0, rinv, lp, 1, 0.0f, gY, lp, P->st));
  return RSVD_OK;
}

// Stage A again (recompute mode): with Q_{j-1} in *qprev, Qt_j in b.wqt and, for j < q, Q_j
// in *qcur -- the forward's kernels and rounds, so the bases are the forward's bit for bit.
rsvd_status_t bw_recompute(rsvd_plan_t P, const void* A, Bw& b, int j, float** qprev, float** qcur) {
  const bool tc = P->opt.precision == RSVD_BF16_TC;
  float* buf[2] = {b.wq0, b.wq1};
  int s;
  int64_t stride;
  TRYS(step_draw(P, tc));
  TRYS(step_pass(P, A, 0, P->omega, false, &s, &stride, P->q == 0));
  TRYS(step_orth(P, P->partial, s, stride, P->m, buf[0], nullptr, P->q == 0));
  const int last = (j < P->q) ? j : j - 1;   // the last Q_i needed
  for (int i = 1; i <= j; ++i) {
    if (tc) TRYS(step_convert(P, buf[(i - 1) & 1], P->m, 0));
    TRYS(step_pass(P, A, 1, buf[(i - 1) & 1], false, &s, &stride));
    TRYS(step_orth(P, P->partial, s, stride, P->n, b.wqt, nullptr, false));
    if (i > last) break;
    if (tc) TRYS(step_convert(P, b.wqt, P->n, 0));
    TRYS(step_pass(P, A, 0, b.wqt, false, &s, &stride, i == P->q));
    TRYS(step_orth(P, P->partial, s, stride, P->m, buf[i & 1], nullptr, i == P->q));
  }
  *qprev = buf[(j - 1) & 1];
  *qcur = (j < P->q) ? buf[j & 1] : P->qbuf;
  return RSVD_OK;
}

rsvd_status_t run_backward(rsvd_plan_t P, const void* A, const float* gU, const float* gS,
                           const float* gV, int add_recon, float* gA) {
  const bool tc = P->opt.precision == RSVD_BF16_TC;
  const bool store = P->opt.recompute == 0;
  const int lp = P->lp, l = P->l, k = P->k, q = P->q;
  const int64_t m = P->m, n = P->n;
  Bw b;
  if (!P->bw) {
    const size_t elems = bw_layout(P, &b, nullptr);
    TRYS(dalloc(P, &P->bw, elems));
  }
  bw_layout(P, &b, P->bw);
  if (tc)
    TRYS(tc_bind_a(&P->tc, A, P->opt.dtype_A == RSVD_BF16X2) == 0 ? RSVD_OK : RSVD_ERR_CUDA);
  const int adt = P->opt.dtype_A == RSVD_F32 ? 0 : (P->opt.dtype_A == RSVD_BF16 ? 1 : 2);
  const float alpha = add_recon ? 2.0f : 0.0f;
  int block = 0;
  // one factor pair (L: m x lp, R: n x lp) of gA = alpha A + sum L R^T
  auto emit = [&](const float* L, const float* R) -> rsvd_status_t {
    if (store) {
      TRY(launch_gather(L, 1, 0, lp, b.lf + (size_t)block * lp, b.kr, m, lp, lp, P->st));
      TRY(launch_gather(R, 1, 0, lp, b.rf + (size_t)block * lp, b.kr, n, lp, lp, P->st));
    } else {
      TRY(launch_lowrank_update(m, n, lp, L, lp, R, lp, A, P->lda, adt, block == 0 ? alpha : 0.0f,
                                block == 0 ? 0.0f : 1.0f, gA, n, P->st));
    }
    ++block;
    return RSVD_OK;
  };
  const size_t l2 = (size_t)lp * lp;
  // clean l x l copies of Ut and W (zero beyond l)
  TRY(cudaMemsetAsync(b.utc, 0, sizeof(float) * l2, P->st));
  TRY(cudaMemsetAsync(b.wc, 0, sizeof(float) * l2, P->st));
  TRY(launch_gather(P->ut(), 1, 0, lp, b.utc, lp, l, l, l, P->st));
  TRY(launch_gather(P->w(), 1, 0, lp, b.wc, lp, l, l, l, P->st));
  // V_B = Q_B W, U_full = Q Ut
  TRY(launch_small_gemm((int)n, lp, lp, 1.0f, P->qtbuf, lp, 0, b.wc, lp, 0, 0.0f, b.vb, lp, P->st));
  TRY(launch_small_gemm((int)m, lp, lp, 1.0f, P->qbuf, lp, 0, b.utc, lp, 0, 0.0f, b.ufull, lp, P->st));
  // the reconstruction loss: P = A V_B, gU_t = gU + 2 S^2 U - 2 S P, gS_t = gS + 1, and the
  // factor (-2 U S, V) of -2 U S V^T
  if (add_recon) {
    TRYS(bw_pass(P, A, 0, b.vb, b.pm));
    TRY(launch_colscale(m, k, lp, b.ufull, lp, P->sig, 0, -2.0f, 0, b.tm, P->st));
    TRY(launch_colscale(n, k, lp, b.vb, lp, nullptr, 0, 1.0f, 0, b.tn, P->st));
    TRYS(emit(b.tm, b.tn));
  }
  TRY(launch_recon_cotangent(m, k, lp, gU, b.ufull, b.pm, P->sig, add_recon, b.gq, P->st));
  TRY(launch_gs_total(gS, k, add_recon, b.gst, P->st));
  // J = Ut^T (Q^T gU_t), K = V_B^T gV (lp x lp, zero beyond column k)
  TRYS(bw_tn(P, m, P->qbuf, b.gq, lp, lp, b.t1));
  TRY(launch_small_gemm(lp, lp, lp, 1.0f, b.utc, lp, 1, b.t1, lp, 0, 0.0f, b.J, lp, P->st));
  if (gV) {
    TRY(launch_colscale(n, k, lp, gV, k, nullptr, 0, 1.0f, 0, b.tn, P->st));   // gV padded to lp columns
    TRYS(bw_tn(P, n, b.vb, b.tn, lp, lp, b.K));
  } else {
    TRY(cudaMemsetAsync(b.K, 0, sizeof(float) * l2, P->st));
  }
  TRY(launch_svd_adjoint(b.J, b.K, P->sig, b.gst, k, l, lp, b.M2, P->st));
  // Z = V_B M2 + gV S^-1
  TRY(launch_small_gemm((int)n, lp, lp, 1.0f, b.vb, lp, 0, b.M2, lp, 0, 0.0f, b.z, lp, P->st));
  if (gV) TRY(launch_colscale(n, k, lp, gV, k, P->sig, 1, 1.0f, 1, b.z, P->st));
  TRYS(emit(b.ufull, b.z));                                    // gA += (Q Ut) Z^T
  // gQ = ((gU_t | 0) + A Z) Ut^T
  TRYS(bw_pass(P, A, 0, b.z, b.tm));
  TRY(launch_colscale(m, lp, lp, b.gq, lp, nullptr, 0, 1.0f, 1, b.tm, P->st));
  TRY(launch_small_gemm((int)m, lp, lp, 1.0f, b.tm, lp, 0, b.utc, lp, 1, 0.0f, b.gq, lp, P->st));
  // Stage A in reverse
  float* q0 = P->basis_q(0);
  for (int j = q; j >= 1; --j) {
    float *qprev, *qcur, *qt;
    if (store) {
      qprev = P->basis_q(j - 1);
      qcur = P->basis_q(j);
      qt = P->basis_qt(j);
    } else {
      TRYS(bw_recompute(P, A, b, j, &qprev, &qcur));
      qt = b.wqt;
    }
    TRYS(bw_qr(P, b, m, qcur, b.gq, P->r_q(j), P->rounds(j == q), b.tm, b.pm));   // gY_j
    TRYS(emit(b.pm, qt));                                       // gA += gY_j Qt_j^T
    TRYS(bw_pass(P, A, 1, b.pm, b.gqt));                        // gQt_j = A^T gY_j
    TRYS(bw_qr(P, b, n, qt, b.gqt, P->r_qt(j), P->rounds(false), b.tn, b.z));     // gYt_j
    TRYS(emit(qprev, b.z));                                     // gA += Q_{j-1} gYt_j^T
    TRYS(bw_pass(P, A, 0, b.z, b.gq));                          // gQ_{j-1} = A gYt_j
    if (j == 1) q0 = qprev;                                     // (recompute mode: still held)
  }
  TRYS(bw_qr(P, b, m, q0, b.gq, P->r_q(0), P->rounds(q == 0), b.tm, b.pm));   // gY_0
  // Omega as the forward multiplied with it (the draw, or the caller's matrix)
  TRYS(step_draw(P, false));
  TRYS(emit(b.pm, P->omega));                                   // gA += gY_0 Omega^T
  if (store)
    TRY(launch_lowrank_update(m, n, block * lp, b.lf, b.kr, b.rf, b.kr, A, P->lda, adt, alpha, 0.0f,
                              gA, n, P->st));
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
  opt->autotune = 1;
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
  if (o.residual_passes != 0 && ((o.residual_passes != 1 && o.residual_passes != 2) || o.dtype_A != RSVD_BF16X2))
    return RSVD_ERR_INVALID_ARG;
  if (o.precision == RSVD_BF16_TC && o.dtype_A == RSVD_F32) return RSVD_ERR_INVALID_ARG;
  if (o.precision != RSVD_PLAIN_FP32 && o.precision != RSVD_BF16_TC) return RSVD_ERR_INVALID_ARG;
  if (o.test_matrix != RSVD_GAUSSIAN && o.test_matrix != RSVD_SRFT && o.test_matrix != RSVD_GSRFT)
    return RSVD_ERR_INVALID_ARG;
  const bool srft = o.test_matrix == RSVD_SRFT || o.test_matrix == RSVD_GSRFT;
  // SRFT: l real columns are l / 2 frequencies from {1 .. n/2 - 1} (Section 4.6 for real A)
  if (srft &&
      ((l & 1) || (n & 1) || l / 2 > n / 2 - 1 || n >= ((int64_t)1 << 24)))
    return RSVD_ERR_INVALID_ARG;
  if (o.small_svd < 0 || o.small_svd > 2) return RSVD_ERR_INVALID_ARG;
  if (o.small_svd == 1 && l > 160) return RSVD_ERR_INVALID_ARG;  // one-CTA Jacobi limit
  if (o.precision == RSVD_BF16_TC && (o.lda % 8) != 0) return RSVD_ERR_INVALID_ARG;  // 16-byte rows
  if (o.host_f32 != 0 && (o.host_f32 != 1 || o.precision != RSVD_BF16_TC)) return RSVD_ERR_INVALID_ARG;
  if (o.srft_fft != 0 && (o.srft_fft != 1 || o.test_matrix != RSVD_SRFT)) return RSVD_ERR_INVALID_ARG;
  if (o.recompute != 0 && o.recompute != 1) return RSVD_ERR_INVALID_ARG;

  rsvd_plan_t P = new (std::nothrow) rsvd_plan_s();
  if (!P) return RSVD_ERR_ALLOC;
  P->m = m; P->n = n; P->k = k; P->p = p; P->q = q; P->l = (int)l;
  P->lp = (int)round_up(l, 16);
  P->lt = P->lpp = 0;
  if (o.single_pass) {
    // Psi: l' columns (Section 5.5 leaves its width open; the default 3 l keeps the system
    // for B^T overdetermined enough on noisy tails)
    int64_t lt = o.psi_cols ? o.psi_cols : std::min<int64_t>(std::min<int64_t>(3 * l, kMaxL), n);
    if (lt < k || lt > kMaxL || lt > n || lt > m) {
      delete P;
      return RSVD_ERR_INVALID_ARG;
    }
    P->lt = (int)lt;
    P->lpp = (int)round_up(lt, 16);
  }
  P->lq = std::max(P->lp, P->lpp);
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
  const int lp = P->lp, lq = P->lq;
  P->splits_n = choose_splits(m, lp, n, P->num_sms);
  P->splits_t = choose_splits(n, lp, m, P->num_sms);
  int64_t part = std::max((int64_t)P->splits_n * m, (int64_t)P->splits_t * n) * lp;
  if (o.single_pass) {
    P->splits_psi = choose_splits(n, P->lpp, m, P->num_sms);
    part = std::max(part, (int64_t)P->splits_psi * n * P->lpp);
  }
  if (o.precision == RSVD_BF16_TC) part = std::max(part, tc_partial_elems(m, n, lq, P->num_sms));
  P->partial_elems = part;
  rsvd_status_t s = RSVD_OK;
  const int nblk = std::max(gram_blocks(m), gram_blocks(n));
  if ((s = dalloc(P, &P->omega, (size_t)n * lp)) != RSVD_OK ||
      (s = dalloc(P, &P->qbuf, (size_t)m * lp)) != RSVD_OK ||
      (s = dalloc(P, &P->qtbuf, (size_t)n * lq)) != RSVD_OK ||
      (s = dalloc(P, &P->tmp1, (size_t)P->maxmn * lq)) != RSVD_OK ||
      (s = dalloc(P, &P->tmp2, (size_t)P->maxmn * lq)) != RSVD_OK ||
      (s = dalloc(P, &P->partial, (size_t)part)) != RSVD_OK ||
      (s = dalloc(P, &P->gpart, (size_t)nblk * lq * lq)) != RSVD_OK ||
      (s = dalloc(P, &P->small, (size_t)24 * lq * lq)) != RSVD_OK ||
      (o.single_pass && (s = dalloc(P, &P->psi, (size_t)m * P->lpp)) != RSVD_OK) ||
      (o.single_pass && (s = dalloc(P, &P->sig2, (size_t)2 * lq)) != RSVD_OK) ||
      (s = dalloc(P, &P->sig, (size_t)lp)) != RSVD_OK ||
      (srft && (s = dalloc(P, &P->srft_freq, (size_t)(l / 2))) != RSVD_OK) ||
      (o.test_matrix == RSVD_GSRFT && (s = dalloc(P, &P->gsrft_perm, gsrft_table_ints(n))) != RSVD_OK) ||
      (s = dalloc(P, &P->status, 4))) {
    free_plan(P);
    return s;
  }
  // the backward's tape (not for the single pass, which has no backward)
  if (!o.single_pass &&
      ((s = dalloc(P, &P->tape_r, (size_t)(2 * q + 1) * 3 * lp * lp)) != RSVD_OK ||
       (q > 0 && !o.recompute && (s = dalloc(P, &P->tape_q, (size_t)q * m * lp)) != RSVD_OK) ||
       (q > 0 && !o.recompute && (s = dalloc(P, &P->tape_qt, (size_t)q * n * lp)) != RSVD_OK))) {
    free_plan(P);
    return s;
  }
  if (o.precision == RSVD_BF16_TC && lq > 128 &&
      (s = dalloc(P, &P->rimg, apply_tc_image_bytes(lq))) != RSVD_OK) {
    free_plan(P);
    return s;
  }
  if (o.precision == RSVD_BF16_TC) {
    const size_t xrows = (size_t)tc_lo_offset(lq) + lq;
    if ((s = dalloc(P, &P->xbf, xrows * (size_t)tc_ld(P->maxmn))) != RSVD_OK ||
        cudaMemsetAsync(P->xbf, 0, xrows * (size_t)tc_ld(P->maxmn) * 2, P->st) != cudaSuccess) {
      free_plan(P);
      return s;
    }
    if (tc_plan_init(&P->tc, m, n, o.lda, lp, P->xbf, P->num_sms) != 0 ||
        (o.single_pass && tc_plan_init(&P->tc2, m, n, o.lda, P->lpp, P->xbf, P->num_sms) != 0)) {
      free_plan(P);
      return RSVD_ERR_CUDA;
    }
    P->tc.status = P->status;
    P->tc2.status = P->status;
  }
  if (srft && (launch_srft_select(seed, n, (int)(l / 2), P->srft_freq, P->st) != cudaSuccess ||
               (o.test_matrix == RSVD_GSRFT &&
                launch_gsrft_prepare(seed, n, P->gsrft_perm, P->st) != cudaSuccess))) {
    cudaGetLastError();
    free_plan(P);
    return RSVD_ERR_CUDA;
  }
  // the signs for the row-transform sketch (the lda must be even for its paired loads)
  // Psi of the single pass (Gaussian, Philox stream 1, l' columns), rounded to bfloat16 for
  // the tensor-core path
  if (o.single_pass &&
      (launch_draw_gaussian(seed, 1u, m, P->lt, P->lpp, P->psi, P->lpp, nullptr, 0, P->st) != cudaSuccess ||
       (o.precision == RSVD_BF16_TC &&
        launch_round_bf16(P->psi, m, P->lpp, P->lpp, P->st) != cudaSuccess))) {
    cudaGetLastError();
    free_plan(P);
    return RSVD_ERR_CUDA;
  }
  if (o.test_matrix == RSVD_SRFT && srft_fft_supported(n) && (o.lda % 2) == 0) {
    if ((s = dalloc(P, &P->srft_signs, (size_t)cdiv(n, 32))) != RSVD_OK) {
      free_plan(P);
      return s;
    }
    if (launch_srft_signs(seed, n, P->srft_signs, P->st) != cudaSuccess) {
      cudaGetLastError();
      free_plan(P);
      return RSVD_ERR_CUDA;
    }
  }
  if (cudaMemsetAsync(P->status, 0, 4 * sizeof(uint32_t), P->st) != cudaSuccess ||
      cudaMemsetAsync(P->small, 0, sizeof(float) * 24 * lq * lq, P->st) != cudaSuccess) {
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
  P->fwd_ok = false;   // the buffers of the last rsvd_svd are reused
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
  P->fwd_ok = false;
  if (P->opt.single_pass) return stage_single_pass(P, A, U, S, V, nullptr, 0);
  TRYS(stage_a(P, A));
  TRYS(stage_b(P, A, U, S, V));
  P->fwd_ok = true;
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
  P->fwd_ok = true;
  return RSVD_OK;
}

namespace {

// bytes from host to device in kCopyStreams pieces, each on its own stream after the work
// already queued on the plan stream; the plan stream then waits for all of them.  (Measured
// with 1 GB from pinned memory: the pieces reach the link's 210 GB/s, where one copy of the
// whole buffer on the plan stream ran at about 130 GB/s.)
rsvd_status_t copy_streams(rsvd_plan_t P) {
  constexpr int NS = rsvd_plan_s::kCopyStreams;
  if (!P->cst[0]) {
    for (int c = 0; c < NS; ++c) TRY(cudaStreamCreateWithFlags(&P->cst[c], cudaStreamNonBlocking));
    for (int c = 0; c <= NS; ++c) TRY(cudaEventCreateWithFlags(&P->cev[c], cudaEventDisableTiming));
  }
  return RSVD_OK;
}

rsvd_status_t copy_in_pieces(rsvd_plan_t P, void* dst, const void* src, size_t bytes) {
  constexpr int NS = rsvd_plan_s::kCopyStreams;
  TRYS(copy_streams(P));
  TRY(cudaEventRecord(P->cev[0], P->st));
  const size_t piece = round_up((int64_t)cdiv((int64_t)bytes, NS), 1 << 16);
  for (int c = 0; c < NS; ++c) {
    const size_t off = (size_t)c * piece;
    if (off >= bytes) break;
    const size_t len = std::min(piece, bytes - off);
    TRY(cudaStreamWaitEvent(P->cst[c], P->cev[0], 0));
    TRY(cudaMemcpyAsync(static_cast<char*>(dst) + off, static_cast<const char*>(src) + off, len,
                        cudaMemcpyHostToDevice, P->cst[c]));
    TRY(cudaEventRecord(P->cev[c + 1], P->cst[c]));
    TRY(cudaStreamWaitEvent(P->st, P->cev[c + 1], 0));
  }
  return RSVD_OK;
}

// host_f32: the float32 A in pieces of rows on the copy streams, each piece split into the
// plan's bfloat16 hi (and lo, m * lda elements further) on its stream once its copy lands
rsvd_status_t copy_split_in_pieces(rsvd_plan_t P, const void* A_host, bool hilo) {
  constexpr int NS = rsvd_plan_s::kCopyStreams;
  TRYS(copy_streams(P));
  TRY(cudaEventRecord(P->cev[0], P->st));
  const int64_t rp = cdiv(P->m, NS);
  __nv_bfloat16* out = static_cast<__nv_bfloat16*>(P->a_dev);
  for (int c = 0; c < NS; ++c) {
    const int64_t r0 = c * rp, r1 = std::min<int64_t>(P->m, r0 + rp);
    if (r0 >= r1) break;
    const size_t len = ((size_t)(r1 - 1 - r0) * P->lda + P->n) * sizeof(float);
    TRY(cudaStreamWaitEvent(P->cst[c], P->cev[0], 0));
    TRY(cudaMemcpyAsync(P->a_f32 + r0 * P->lda, static_cast<const float*>(A_host) + r0 * P->lda, len,
                        cudaMemcpyHostToDevice, P->cst[c]));
    TRY(launch_split_bf16(P->a_f32 + r0 * P->lda, r1 - r0, P->n, P->lda, out + r0 * P->lda, P->lda,
                          hilo ? 1 : 0, P->cst[c], P->m * P->lda));
    TRY(cudaEventRecord(P->cev[c + 1], P->cst[c]));
    TRY(cudaStreamWaitEvent(P->st, P->cev[c + 1], 0));
  }
  return RSVD_OK;
}

}  // namespace

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
    // float32 in, the plan's bfloat16 storage (hi, and lo m * lda elements further) out,
    // piece by piece, each split while the next ones are still being copied
    TRYS(copy_split_in_pieces(P, A_host, hilo));
  } else {
    TRYS(copy_in_pieces(P, P->a_dev, A_host, abytes));
  }
  TRYS(rsvd_svd(P, P->a_dev, P->u_dev, P->s_dev, P->v_dev));
  TRY(cudaMemcpyAsync(U_host, P->u_dev, sizeof(float) * P->m * P->k, cudaMemcpyDeviceToHost, P->st));
  TRY(cudaMemcpyAsync(S_host, P->s_dev, sizeof(float) * P->k, cudaMemcpyDeviceToHost, P->st));
  TRY(cudaMemcpyAsync(V_host, P->v_dev, sizeof(float) * P->n * P->k, cudaMemcpyDeviceToHost, P->st));
  return take_status(P);
}

rsvd_status_t rsvd_svd_backward(rsvd_plan_t P, const void* A, const float* gU, const float* gS,
                                const float* gV, int32_t add_recon, float* gA) {
  TRYS(check_plan(P));
  if (!A || !gA || (add_recon != 0 && add_recon != 1)) return RSVD_ERR_INVALID_ARG;
  if (P->opt.single_pass) return RSVD_ERR_UNSUPPORTED;
  if (!P->fwd_ok) return RSVD_ERR_INVALID_ARG;   // needs the state of an rsvd_svd call on A
  return run_backward(P, A, gU, gS, gV, add_recon, gA);
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
  P->fwd_ok = false;   // the buffers of the last rsvd_svd are reused
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

rsvd_status_t rsvd_wait_selftest(rsvd_plan_t P, uint32_t spins) {
  TRYS(check_plan(P));
  if (spins == 0) return RSVD_ERR_INVALID_ARG;
  // status word 3 is never written by any kernel: the wait can only run out
  TRY(launch_wait_selftest(P->status + 3, spins, P->status, P->st));
  return RSVD_OK;
}

void rsvd_debug_fail_alloc(int32_t after) { g_fail_alloc_after.store(after < 0 ? -1 : after); }

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
  P->fwd_ok = false;   // the buffers of the last rsvd_svd are reused
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
  TRYS(step_pass(P, A, transpose, xin, false, &s, &stride, true));
  TRY(launch_gather(P->partial, s, stride, P->lp, Y, P->l, my, P->l, P->l, P->st));
  return RSVD_OK;
}

// Hermitian Stage B (Section 5.3, 5.4) after Stage A: B1 = A Q (one pass, the basis as a
// hi + lo pair on the tensor cores), B = Q^T B1 symmetrised; Algorithm 5.3 takes the
// eigenpairs of B from its SVD (the sign of each eigenvalue from its pair of singular
// vectors) and lifts U = Q V; Algorithm 5.5 factors B = C^T C (Cholesky, with the pivot
// floor), F = B1 C^-1, and takes F = U S W^T through Cholesky QR and Jacobi (U = Q_F Ut),
// Lambda = S^2.
rsvd_status_t run_eig(rsvd_plan_t P, const void* A, int method, float* U, float* Lambda) {
  const bool tc = P->opt.precision == RSVD_BF16_TC;
  const int lp = P->lp, l = P->l, k = P->k;
  TRYS(stage_a(P, A));
  int s;
  int64_t stride;
  if (tc) TRYS(step_convert(P, P->qbuf, P->m, 1));
  TRYS(step_pass(P, A, 0, P->qbuf, true, &s, &stride));             // B1 = A Q
  TRY(launch_gather(P->partial, s, stride, lp, P->tmp1, lp, P->m, lp, lp, P->st));
  {
    Step sp(P, RSVD_STEP_SMALL_SVD);
    sp.launched(4);
    TRYS(bw_tn(P, P->m, P->qbuf, P->tmp1, lp, lp, P->sq()));           // B = Q^T B1
    TRY(launch_symmetrize(P->sq(), l, lp, P->st));
    if (method == RSVD_EIG_DIRECT) {
      TRY(launch_jacobi_svd(P->sq(), lp, 0, l, lp, P->ut(), P->sig, P->w(), P->lbuf(), P->status,
                            P->status + 1, P->st, P->opt.small_svd));
      TRY(launch_eig_values(P->ut(), P->w(), P->sig, l, lp, k, 0, Lambda, P->st));
    }
  }
  if (method == RSVD_EIG_DIRECT) {
    Step sp(P, RSVD_STEP_LIFT);
    sp.launched();
    TRY(launch_gemm_f32(0, P->m, k, lp, P->qbuf, lp, P->ut(), lp, U, k, 1, 0, P->st));
    return RSVD_OK;
  }
  // Nystrom: B = C^T C, F = B1 C^-1, F = Q_F R_F, R_F = Ut S W^T, U = Q_F Ut, Lambda = S^2
  {
    Step sp(P, RSVD_STEP_ORTH);
    sp.launched(2);
    TRY(launch_cholesky(P->sq(), l, lp, 0, P->lbuf(), P->rtmp(), P->rinv(), nullptr, 0, P->status,
                        P->st));
    TRY(launch_gemm_f32(0, P->m, lp, lp, P->tmp1, lp, P->rinv(), lp, P->tmp2, lp, 1, 0, P->st));
  }
  TRYS(step_orth(P, P->tmp2, 1, P->m * lp, P->m, P->qtbuf, P->racc()));
  {
    Step sp(P, RSVD_STEP_SMALL_SVD);
    sp.launched(2);
    TRY(launch_jacobi_svd(P->racc(), lp, 0, l, lp, P->ut(), P->sig, P->w(), P->lbuf(), P->status,
                          P->status + 1, P->st, P->opt.small_svd));
    TRY(launch_eig_values(P->ut(), P->w(), P->sig, l, lp, k, 1, Lambda, P->st));
  }
  Step sp(P, RSVD_STEP_LIFT);
  sp.launched();
  TRY(launch_gemm_f32(0, P->m, k, lp, P->qtbuf, lp, P->ut(), lp, U, k, 1, 0, P->st));
  return RSVD_OK;
}

// The row ID of res (m x lp, ld lp, overwritten): pivots and coefficients in the row ID
// workspace, then Linv = L^-1 (lower, ld lp) in sp(1) from Lt = C[J]^T (sp(0)).
struct Re {
  float* coef;
  float* cand;
  int* piv;
  unsigned* bar;
};

rsvd_status_t re_workspace(rsvd_plan_t P, Re* w) {
  const int lp = P->lp;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(P->num_sms, cdiv(P->m, 64)));
  const size_t cm = (size_t)P->m * lp, cc = id_cand_floats(grid, lp);
  const size_t coff = (cm + 63) & ~size_t(63), poff = coff + ((cc + 63) & ~size_t(63));
  if (!P->re) {
    TRYS(dalloc(P, &P->re, poff + (size_t)lp + 64));
    P->re_grid = grid;
  }
  w->coef = P->re;
  w->cand = P->re + coff;
  w->piv = reinterpret_cast<int*>(P->re + poff);
  w->bar = reinterpret_cast<unsigned*>(P->re + poff + lp);
  return RSVD_OK;
}

rsvd_status_t step_row_id(rsvd_plan_t P, float* res, Re* w) {
  const int lp = P->lp, l = P->l;
  TRYS(re_workspace(P, w));
  {
    Step sp(P, RSVD_STEP_ID);
    sp.launched();
    TRY(cudaMemsetAsync(w->coef, 0, sizeof(float) * (size_t)P->m * lp, P->st));
    TRY(cudaMemsetAsync(w->bar, 0, sizeof(unsigned), P->st));
    TRY(launch_id_pivot(res, P->m, l, lp, w->coef, w->piv, w->cand, w->bar, P->status, P->re_grid,
                        P->st));
  }
  Step sp(P, RSVD_STEP_SMALL_SVD);
  sp.launched(3);
  TRY(launch_id_lt(w->coef, w->piv, l, lp, P->sp(0), P->st));
  TRY(launch_trinv_upper(P->sp(0), l, lp, P->sp(2), P->st));      // L^-T
  TRY(launch_transpose_square(P->sp(2), lp, P->sp(1), P->st));    // L^-1
  return RSVD_OK;
}

// Algorithm 5.2 after Stage A: the ID of Q (in place in qbuf), A[J]^T = W R, Z = C L^-1 R^T,
// Z = Q_Z R_Z, R_Z = Ut S Vt^T, U = Q_Z Ut, V = W Vt.
rsvd_status_t run_row_extraction(rsvd_plan_t P, const void* A, float* U, float* S, float* V) {
  const int lp = P->lp, l = P->l, k = P->k;
  TRYS(stage_a(P, A));
  Re w;
  TRYS(step_row_id(P, P->qbuf, &w));
  {
    Step sp(P, RSVD_STEP_CONVERT);
    sp.launched();
    const int adt = P->opt.dtype_A == RSVD_F32 ? 0 : (P->opt.dtype_A == RSVD_BF16 ? 1 : 2);
    TRY(launch_gather_rows_t(adt, A, P->lda, P->m, P->n, w.piv, l, lp, P->partial, P->st));
  }
  TRYS(step_orth(P, P->partial, 1, P->n * lp, P->n, P->qtbuf, P->racc()));   // A[J]^T = W R
  {
    Step sp(P, RSVD_STEP_SMALL_SVD);
    sp.launched(2);
    TRY(cudaMemsetAsync(P->sp(3), 0, sizeof(float) * (size_t)lp * lp, P->st));
    TRY(launch_small_gemm(l, l, l, 1.f, P->sp(1), lp, 0, P->racc(), lp, 1, 0.f, P->sp(3), lp, P->st));
  }
  {
    Step sp(P, RSVD_STEP_LIFT);
    sp.launched();
    TRY(launch_gemm_f32(0, P->m, lp, lp, w.coef, lp, P->sp(3), lp, P->tmp2, lp, 1, 0, P->st));  // Z
  }
  TRYS(step_orth(P, P->tmp2, 1, P->m * lp, P->m, P->qbuf, P->racc()));
  {
    Step sp(P, RSVD_STEP_SMALL_SVD);
    sp.launched();
    TRY(launch_jacobi_svd(P->racc(), lp, 0, l, lp, P->ut(), P->sig, P->w(), P->lbuf(), P->status,
                          P->status + 1, P->st, P->opt.small_svd));
  }
  Step sp(P, RSVD_STEP_LIFT);
  sp.launched(2);
  TRY(launch_gemm_f32(0, P->m, k, lp, P->qbuf, lp, P->ut(), lp, U, k, 1, 0, P->st));
  TRY(launch_gemm_f32(0, P->n, k, lp, P->qtbuf, lp, P->w(), lp, V, k, 1, 0, P->st));
  TRY(cudaMemcpyAsync(S, P->sig, sizeof(float) * k, cudaMemcpyDeviceToDevice, P->st));
  return RSVD_OK;
}

rsvd_status_t rsvd_row_id(rsvd_plan_t P, const float* Y, int64_t ldy, int32_t* J, float* X, int64_t ldx) {
  TRYS(check_plan(P));
  if (!Y || !J || !X || ldy < P->l || ldx < P->l) return RSVD_ERR_INVALID_ARG;
  P->fwd_ok = false;
  TRY(launch_gather(Y, 1, 0, ldy, P->tmp1, P->lp, P->m, P->l, P->lp, P->st));
  Re w;
  TRYS(step_row_id(P, P->tmp1, &w));
  Step sp(P, RSVD_STEP_LIFT);
  sp.launched();
  TRY(launch_gemm_f32(0, P->m, P->l, P->lp, w.coef, P->lp, P->sp(1), P->lp, X, ldx, 1, 0, P->st));
  TRY(cudaMemcpyAsync(J, w.piv, sizeof(int32_t) * P->l, cudaMemcpyDeviceToDevice, P->st));
  return RSVD_OK;
}

rsvd_status_t rsvd_svd_row_extraction(rsvd_plan_t P, const void* A, float* U, float* S, float* V) {
  TRYS(check_plan(P));
  if (!A || !U || !S || !V) return RSVD_ERR_INVALID_ARG;
  if (P->opt.single_pass) return RSVD_ERR_UNSUPPORTED;
  P->fwd_ok = false;
  return run_row_extraction(P, A, U, S, V);
}

rsvd_status_t rsvd_eig(rsvd_plan_t P, const void* A, int32_t method, float* U, float* Lambda) {
  TRYS(check_plan(P));
  if (!A || !U || !Lambda || P->m != P->n ||
      (method != RSVD_EIG_DIRECT && method != RSVD_EIG_NYSTROM))
    return RSVD_ERR_INVALID_ARG;
  if (P->opt.single_pass) return RSVD_ERR_UNSUPPORTED;
  P->fwd_ok = false;
  return run_eig(P, A, method, U, Lambda);
}

rsvd_status_t rsvd_range_finder_adaptive(rsvd_plan_t P, const void* A, float eps, int32_t block,
                                         float* Q, int64_t ldq, int32_t* rank, float* estimate) {
  TRYS(check_plan(P));
  if (!A || !Q || !rank || !(eps > 0.0f) || block < 16 || block % 16 || block > P->l ||
      ldq < P->l)
    return RSVD_ERR_INVALID_ARG;
  if (P->opt.single_pass) return RSVD_ERR_UNSUPPORTED;
  P->fwd_ok = false;
  return run_adaptive(P, A, eps, block, Q, ldq, rank, estimate);
}

rsvd_status_t rsvd_sketch_srft(rsvd_plan_t P, const void* A, float* Y) {
  TRYS(check_plan(P));
  if (!A || !Y) return RSVD_ERR_INVALID_ARG;
  if (P->opt.test_matrix != RSVD_SRFT || !P->srft_signs) return RSVD_ERR_UNSUPPORTED;
  P->fwd_ok = false;
  TRYS(step_srft_fft(P, A, P->partial));
  TRY(launch_gather(P->partial, 1, 0, P->lp, Y, P->l, P->m, P->l, P->l, P->st));
  return RSVD_OK;
}

rsvd_status_t rsvd_orthonormalize(rsvd_plan_t P, int64_t rows, float* Y, float* R) {
  TRYS(check_plan(P));
  P->fwd_ok = false;   // the buffers of the last rsvd_svd are reused
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
  P->fwd_ok = false;   // the buffers of the last rsvd_svd are reused
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
