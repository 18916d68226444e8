// Batched C ABI: one plan for many small matrices (l = k + p <= 32), each step of the
// randomized SVD (Algorithm 4.4 + Algorithm 5.1) one launch over the whole batch, and
// the gradient of the batched reconstruction loss through that map (test matrices fixed).
// Every pass after the first carries its float32 operand as a bfloat16 hi/lo pair (the
// passes are bound by reading A, so the doubled MMA width costs nothing measurable), and
// Omega is drawn as bfloat16 values: the map differentiated by the backward pass is the
// float32 map on the bfloat16 A with a bfloat16 Omega.
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "kernels_batched.cuh"
#include "sketch_tc.cuh"

struct rsvd_batched_plan_s {
  int nb = 0, k = 0, p = 0, q = 0, l = 0;
  uint64_t seed = 0;
  rsvd_options_t opt{};
  cudaStream_t st = nullptr;
  int num_sms = 0;
  std::vector<int64_t> m, n, lda;
  int64_t sum_m = 0, sum_n = 0, xm_total = 0, xn_total = 0;
  int64_t max_m = 0, max_n = 0;
  // device index arrays
  int64_t* d_roff_m = nullptr;   // nb + 1
  int64_t* d_roff_n = nullptr;   // nb + 1
  int64_t* d_xoff_m = nullptr;   // nb
  int64_t* d_xoff_n = nullptr;   // nb
  int64_t* d_m = nullptr;        // nb
  int64_t* d_n = nullptr;        // nb
  int2* d_units0 = nullptr;      // (b, row tile of m_b)
  int2* d_units1 = nullptr;      // (b, row tile of n_b)
  int nunits0 = 0, nunits1 = 0;
  int2* d_qunits_m = nullptr;     // Cholesky-QR units (b, 128-row tile) in matrix order, m side
  int2* d_qunits_n = nullptr;     // the same on the n side
  int* d_ustart_m = nullptr;      // nb + 1: the first unit of each matrix
  int* d_ustart_n = nullptr;
  int nq_m = 0, nq_n = 0;
  float* qpart = nullptr;         // max(nq_m, nq_n) x 32 x 32 Gram partials
  // tensor maps of A_b (mode 0 boxes, then mode 1 boxes), device copy + the bound pointers
  unsigned char* d_maps = nullptr;
  std::vector<unsigned char> h_maps;
  std::vector<const void*> a_bound;
  alignas(64) unsigned char map_x_m[128];   // operand with K = sum of padded m_b (32 rows)
  alignas(64) unsigned char map_x_n[128];   // operand with K = sum of padded n_b (32 rows)
  alignas(64) unsigned char map_x_m2[128];  // the same with the lo half (64 rows)
  alignas(64) unsigned char map_x_n2[128];
  // workspace
  __nv_bfloat16* xbf = nullptr;   // 2 LP x max(xm_total, xn_total): hi rows, then lo rows
  float* omega = nullptr;         // sum_n x LP
  float* ym = nullptr;            // sum_m x LP   pass outputs (m side)
  float* yn = nullptr;            // sum_n x LP   pass outputs (n side)
  std::vector<float*> qm;         // q + 1 bases on the m side (Q_0 .. Q_q)
  std::vector<float*> qn;         // q bases on the n side (Qt_1 .. Qt_q)
  std::vector<float*> rm, rn;     // their R factors, nb x LP x LP each
  float* qb = nullptr;            // sum_n x LP   Q_B
  float* rb = nullptr;            // nb x LP x LP R_B
  float* ub = nullptr;            // nb x LP x LP singular vectors of R_B^T (left)
  float* wb = nullptr;            // nb x LP x LP (right)
  float* sig = nullptr;           // nb x LP
  uint32_t* status = nullptr;     // [0] status bits, [1] Jacobi sweeps
  // backward workspace
  int kr = 0;                     // 32 (2q + 2) columns of the low-rank factors of dL/dA
  float* lbuf = nullptr;          // sum_m x kr
  float* rbuf = nullptr;          // sum_n x kr
  __nv_bfloat16* lplanes = nullptr;  // 3 x sum_m x kr: the bfloat16 split of lbuf (h, m, t)
  __nv_bfloat16* rplanes = nullptr;  // 3 x sum_n x kr
  alignas(64) unsigned char map_lp[128];  // tensor maps of the planes (box 64 x 128)
  alignas(64) unsigned char map_rp[128];
  float* gm = nullptr;            // sum_m x LP
  float* pm = nullptr;            // sum_m x LP
  float* gn = nullptr;            // sum_n x LP
  float* nmat = nullptr;          // nb x LP x LP
  float* rinv = nullptr;          // nb x LP x LP
  int4* d_units_f = nullptr;      // (b, row tile, column tile) of dL/dA, bwd_final_tile() square
  int nunits_f = 0;
  int64_t* d_lda = nullptr;
  const void** d_aptr = nullptr;
  float** d_gptr = nullptr;
  size_t ws_bytes = 0;
  std::vector<void*> allocs;
  // CUDA graphs of the forward and of the backward for one binding of the pointers (the
  // A_b, and U, S, V or the gA_b): every launch of a call replayed as one graph launch
  cudaGraphExec_t g_fwd = nullptr, g_bwd = nullptr;
  // pass configuration per (mode, fold): pipeline stages and CTAs per SM, picked by the
  // autotuner on the first call (tuned = true) or read from its JSON cache
  int cfg_stages[4] = {rsvd::kBatchedStages, rsvd::kBatchedStages, rsvd::kBatchedStages,
                       rsvd::kBatchedStages};
  int cfg_ctas[4] = {1, 1, 1, 1};
  bool tuned = false;
  std::vector<const void*> g_fwd_a, g_bwd_a;
  std::vector<float*> g_bwd_g;
  const float *g_u = nullptr, *g_s = nullptr, *g_v = nullptr;
  bool use_graph = true;
};

namespace rsvd {
namespace {

constexpr int LP = kBatchedLP;

#define BTRY(expr)                                \
  do {                                            \
    cudaError_t _e = (expr);                      \
    if (_e != cudaSuccess) return RSVD_ERR_CUDA;  \
  } while (0)
#define BTRYS(expr)                 \
  do {                              \
    rsvd_status_t _s = (expr);      \
    if (_s != RSVD_OK) return _s;   \
  } while (0)

template <typename T>
rsvd_status_t balloc(rsvd_batched_plan_t P, T** ptr, size_t elems) {
  *ptr = nullptr;
  const size_t bytes = std::max<size_t>(elems, 1) * sizeof(T);
  if (cudaMalloc(reinterpret_cast<void**>(ptr), bytes) != cudaSuccess) {
    cudaGetLastError();
    return RSVD_ERR_ALLOC;
  }
  P->allocs.push_back(*ptr);
  P->ws_bytes += bytes;
  return RSVD_OK;
}

void bfree(rsvd_batched_plan_t P) {
  if (!P) return;
  if (P->g_fwd) cudaGraphExecDestroy(P->g_fwd);
  if (P->g_bwd) cudaGraphExecDestroy(P->g_bwd);
  for (void* a : P->allocs) cudaFree(a);
  delete P;
}

template <typename T>
rsvd_status_t upload(rsvd_batched_plan_t P, T** dst, const std::vector<T>& src) {
  BTRYS(balloc(P, dst, src.size()));
  BTRY(cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
  return RSVD_OK;
}

// units of a pass, heaviest first (largest K), so that the round-robin deal to CTAs balances
// 128-row units of every matrix in matrix order and the first unit of each matrix
std::vector<int2> make_qr_units(const std::vector<int64_t>& rows, std::vector<int>* ustart) {
  std::vector<int2> u;
  ustart->assign(rows.size() + 1, 0);
  for (size_t b = 0; b < rows.size(); ++b) {
    (*ustart)[b] = (int)u.size();
    for (int64_t t = 0; t < cdiv(rows[b], 128); ++t) u.push_back(make_int2((int)b, (int)t));
  }
  (*ustart)[rows.size()] = (int)u.size();
  return u;
}

std::vector<int2> make_units(const std::vector<int64_t>& rows, const std::vector<int64_t>& kext) {
  std::vector<int> order(rows.size());
  for (size_t b = 0; b < rows.size(); ++b) order[b] = (int)b;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return kext[a] > kext[c]; });
  std::vector<int2> u;
  for (int b : order)
    for (int64_t t = 0; t < cdiv(rows[b], 128); ++t) u.push_back(make_int2(b, (int)t));
  return u;
}

rsvd_status_t bind_maps(rsvd_batched_plan_t P, const void* const* A) {
  bool same = true;
  for (int b = 0; b < P->nb && same; ++b) same = (P->a_bound[b] == A[b]);
  if (same) return RSVD_OK;
  for (int b = 0; b < P->nb; ++b) {
    if (!A[b] || (reinterpret_cast<uintptr_t>(A[b]) & 15)) return RSVD_ERR_INVALID_ARG;
    unsigned char* m0 = P->h_maps.data() + (size_t)b * 128;
    unsigned char* m1 = P->h_maps.data() + (size_t)(P->nb + b) * 128;
    if (tc_encode_2d(m0, A[b], P->n[b], P->m[b], P->lda[b], 64, 128) ||
        tc_encode_2d(m1, A[b], P->n[b], P->m[b], P->lda[b], 64, 64))
      return RSVD_ERR_CUDA;
  }
  BTRY(cudaMemcpyAsync(P->d_maps, P->h_maps.data(), P->h_maps.size(), cudaMemcpyHostToDevice, P->st));
  for (int b = 0; b < P->nb; ++b) P->a_bound[b] = A[b];
  return RSVD_OK;
}

// Y = A X (mode 0: X on the n side, Y on the m side) or Y = A^T X (mode 1); fold: the
// operand holds hi and lo halves
rsvd_status_t bpass_cfg(rsvd_batched_plan_t P, int mode, int fold, float* y, int stages, int ctas) {
  const void* maps = P->d_maps + (mode ? (size_t)P->nb * 128 : 0);
  const int grid = P->num_sms * ctas;
  if (mode == 0)
    BTRY(launch_batched_tc(0, fold, maps, fold ? P->map_x_n2 : P->map_x_n, P->d_units0, P->nunits0,
                           P->d_n, P->d_m, P->d_xoff_n, P->d_roff_m, y, grid, P->status, P->st, stages));
  else
    BTRY(launch_batched_tc(1, fold, maps, fold ? P->map_x_m2 : P->map_x_m, P->d_units1, P->nunits1,
                           P->d_m, P->d_n, P->d_xoff_m, P->d_roff_n, y, grid, P->status, P->st, stages));
  return RSVD_OK;
}

rsvd_status_t bpass(rsvd_batched_plan_t P, int mode, int fold, float* y) {
  const int c = 2 * mode + fold;
  return bpass_cfg(P, mode, fold, y, P->cfg_stages[c], P->cfg_ctas[c]);
}

// ---- autotuner of the grouped pass ------------------------------------------------------
// Candidates (pipeline stages, CTAs per SM): deep pipelines with one CTA per SM, or shallower
// ones with two CTAs sharing an SM (more units in flight: the batch's units are short, at
// most 32 k tiles).  Each (mode, fold) pass is timed with CUDA events on the plan's stream
// on the caller's matrices (two launches per candidate, the second timed) and the fastest
// kept.  Choices are cached per shape class in the JSON file named by RSVD_TUNE_CACHE (an
// object of "key": [stages, ctas, ...] entries), so a later plan of the same class skips
// the timing.
constexpr int kTuneCand[][2] = {{8, 1}, {6, 1}, {4, 2}, {3, 2}};

std::string tune_key(rsvd_batched_plan_t P) {
  char buf[160];
  snprintf(buf, sizeof buf, "batched_pass b%d m%lld n%lld l%d sms%d", P->nb, (long long)P->sum_m,
           (long long)P->sum_n, P->l, P->num_sms);
  return buf;
}

bool tune_cache_read(const std::string& key, int* stages, int* ctas) {
  const char* path = getenv("RSVD_TUNE_CACHE");
  if (!path || !path[0]) return false;
  FILE* f = fopen(path, "rb");
  if (!f) return false;
  std::string text;
  char chunk[4096];
  size_t got;
  while ((got = fread(chunk, 1, sizeof chunk, f)) > 0) text.append(chunk, got);
  fclose(f);
  const std::string pat = "\"" + key + "\"";
  const size_t at = text.find(pat);
  if (at == std::string::npos) return false;
  const size_t lb = text.find('[', at + pat.size());
  if (lb == std::string::npos) return false;
  int v[8];
  if (sscanf(text.c_str() + lb, "[%d,%d,%d,%d,%d,%d,%d,%d]", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5],
             &v[6], &v[7]) != 8)
    return false;
  for (int c = 0; c < 4; ++c) {
    if (v[2 * c] < 2 || v[2 * c] > kBatchedStages || v[2 * c + 1] < 1 || v[2 * c + 1] > 2) return false;
    stages[c] = v[2 * c];
    ctas[c] = v[2 * c + 1];
  }
  return true;
}

void tune_cache_write(const std::string& key, const int* stages, const int* ctas) {
  const char* path = getenv("RSVD_TUNE_CACHE");
  if (!path || !path[0]) return;
  std::string text;
  if (FILE* f = fopen(path, "rb")) {
    char chunk[4096];
    size_t got;
    while ((got = fread(chunk, 1, sizeof chunk, f)) > 0) text.append(chunk, got);
    fclose(f);
  }
  // keep the other keys' entries (one per line), replace this key's
  std::string out = "{\n";
  size_t pos = 0;
  bool first = true;
  while ((pos = text.find('"', pos)) != std::string::npos) {
    const size_t end = text.find('"', pos + 1);
    const size_t eol = text.find(']', end);
    if (end == std::string::npos || eol == std::string::npos) break;
    const std::string k = text.substr(pos + 1, end - pos - 1);
    if (k != key) {
      out += first ? "  " : ",\n  ";
      out += text.substr(pos, eol + 1 - pos);
      first = false;
    }
    pos = eol + 1;
  }
  char entry[256];
  snprintf(entry, sizeof entry, "%s\"%s\": [%d,%d,%d,%d,%d,%d,%d,%d]\n}\n", first ? "  " : ",\n  ",
           key.c_str(), stages[0], ctas[0], stages[1], ctas[1], stages[2], ctas[2], stages[3], ctas[3]);
  out += entry;
  const std::string tmp = std::string(path) + ".tmp";
  if (FILE* f = fopen(tmp.c_str(), "wb")) {
    fwrite(out.data(), 1, out.size(), f);
    fclose(f);
    rename(tmp.c_str(), path);
  }
}

rsvd_status_t autotune(rsvd_batched_plan_t P) {
  const std::string key = tune_key(P);
  if (tune_cache_read(key, P->cfg_stages, P->cfg_ctas)) {
    P->tuned = true;
    return RSVD_OK;
  }
  cudaEvent_t e0, e1;
  BTRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return RSVD_ERR_CUDA;
  }
  rsvd_status_t st = RSVD_OK;
  for (int c = 0; c < 4 && st == RSVD_OK; ++c) {
    const int mode = c >> 1, fold = c & 1;
    float* y = mode ? P->yn : P->ym;
    float best = 1e30f;
    for (const auto& cand : kTuneCand) {
      float ms = 0.0f;
      if ((st = bpass_cfg(P, mode, fold, y, cand[0], cand[1])) != RSVD_OK) break;
      if (cudaEventRecord(e0, P->st) != cudaSuccess ||
          (st = bpass_cfg(P, mode, fold, y, cand[0], cand[1])) != RSVD_OK ||
          cudaEventRecord(e1, P->st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        if (st == RSVD_OK) st = RSVD_ERR_CUDA;
        break;
      }
      if (ms < best) {
        best = ms;
        P->cfg_stages[c] = cand[0];
        P->cfg_ctas[c] = cand[1];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != RSVD_OK) return st;
  P->tuned = true;
  tune_cache_write(key, P->cfg_stages, P->cfg_ctas);
  return RSVD_OK;
}

rsvd_status_t to_operand(rsvd_batched_plan_t P, const float* q, bool m_side, int split) {
  BTRY(launch_batched_to_bf16t(q, m_side ? P->d_roff_m : P->d_roff_n, P->nb, m_side ? P->sum_m : P->sum_n,
                               P->xbf, std::max(P->xm_total, P->xn_total),
                               m_side ? P->d_xoff_m : P->d_xoff_n, split, P->st));
  return RSVD_OK;
}

// The caller (rsvd_batched_svd) has bound the maps of the A_b.
rsvd_status_t bforward(rsvd_batched_plan_t P, const void* const* A, float* U, float* S, float* V) {
  (void)A;
  const int64_t ldx = std::max(P->xm_total, P->xn_total);
  // A basis that only feeds the next pass needs to span its sample, not to be orthonormal to
  // working precision: it gets the shifted round and one plain one, final bases every round
  // (the rule of the single-matrix path).
  const int rounds = P->opt.orth_rounds;
  const int rounds_mid = std::min(rounds, 2);
  const int shift = rounds >= 3 ? 1 : 0;
  BTRY(launch_batched_draw(P->seed, P->d_roff_n, P->nb, P->sum_n, P->l, P->omega, P->xbf, ldx,
                           P->d_xoff_n, P->st));
  BTRYS(bpass(P, 0, 0, P->ym));                                                  // Y_0 = A Omega
  // every basis of Stage A is also written by its last Cholesky-QR round as the next pass's
  // operand (transposed bfloat16 hi + lo)
  BTRY(launch_batched_cholqr(P->ym, P->qm[0], P->d_roff_m, P->nb, P->l, P->q == 0 ? rounds : rounds_mid, shift,
                             P->rm[0], P->rinv, P->d_qunits_m, P->nq_m, P->d_ustart_m, P->qpart, P->status,
                             P->st, P->xbf, ldx, P->d_xoff_m, 1));
  for (int j = 1; j <= P->q; ++j) {
    BTRYS(bpass(P, 1, 1, P->yn));                                                // A^T Q_{j-1}
    BTRY(launch_batched_cholqr(P->yn, P->qn[j - 1], P->d_roff_n, P->nb, P->l, rounds_mid, shift, P->rn[j - 1],
                               P->rinv, P->d_qunits_n, P->nq_n, P->d_ustart_n, P->qpart, P->status, P->st,
                               P->xbf, ldx, P->d_xoff_n, 1));
    BTRYS(bpass(P, 0, 1, P->ym));                                                // A Qt_j
    BTRY(launch_batched_cholqr(P->ym, P->qm[j], P->d_roff_m, P->nb, P->l, j == P->q ? rounds : rounds_mid, shift,
                               P->rm[j], P->rinv, P->d_qunits_m, P->nq_m, P->d_ustart_m, P->qpart, P->status,
                               P->st, P->xbf, ldx, P->d_xoff_m, 1));
  }
  float* Q = P->qm[P->q];
  BTRYS(bpass(P, 1, 1, P->yn));                                                  // B^T = A^T Q (split Q)
  BTRY(launch_batched_cholqr(P->yn, P->qb, P->d_roff_n, P->nb, P->l, rounds, shift, P->rb, P->rinv,
                             P->d_qunits_n, P->nq_n, P->d_ustart_n, P->qpart, P->status, P->st));
  BTRY(launch_batched_jacobi(P->rb, 1, P->l, P->nb, P->ub, P->sig, P->wb, P->status, P->status + 1, P->st));
  if (U) BTRY(launch_batched_lift(Q, P->d_roff_m, P->nb, P->max_m, P->l, P->ub, P->k, P->k, U, P->k, P->st));
  if (V) BTRY(launch_batched_lift(P->qb, P->d_roff_n, P->nb, P->max_n, P->l, P->wb, P->k, P->k, V, P->k, P->st));
  if (S)
    BTRY(cudaMemcpy2DAsync(S, sizeof(float) * P->k, P->sig, sizeof(float) * LP, sizeof(float) * P->k,
                           P->nb, cudaMemcpyDeviceToDevice, P->st));
  return RSVD_OK;
}

// dL/dY from dL/dQ for Y = Q R (rows of one side): N, R^-1 per matrix, then per row
rsvd_status_t qr_back(rsvd_batched_plan_t P, const float* Q, const float* gQ, const float* R, bool m_side,
                      float* gY) {
  const int64_t* roff = m_side ? P->d_roff_m : P->d_roff_n;
  BTRY(launch_bwd_qr_small(Q, gQ, roff, m_side ? P->d_qunits_m : P->d_qunits_n, m_side ? P->nq_m : P->nq_n,
                           m_side ? P->d_ustart_m : P->d_ustart_n, P->nb, P->l, R, P->qpart, P->nmat, P->rinv,
                           P->st));
  BTRY(launch_bwd_qr_apply(Q, gQ, roff, m_side ? P->d_qunits_m : P->d_qunits_n, m_side ? P->nq_m : P->nq_n,
                           P->l, P->nmat, P->rinv, gY, P->st));
  return RSVD_OK;
}

// The caller (rsvd_batched_svd_backward) has bound the maps and copied the pointer arrays.
rsvd_status_t bbackward(rsvd_batched_plan_t P, const void* const* A, float* const* gA) {
  (void)A;
  (void)gA;
  const int kr = P->kr;
  // V = Q_B W_k (n side) is the first right factor and the operand of A V
  BTRY(launch_batched_lift(P->qb, P->d_roff_n, P->nb, P->max_n, P->l, P->wb, LP, P->k, P->gn, LP, P->st));
  BTRY(launch_copy_block(P->gn, P->sum_n, P->rbuf, kr, 0, P->st));
  BTRYS(to_operand(P, P->gn, false, 1));
  BTRYS(bpass(P, 0, 1, P->pm));                                                  // A V
  // dL/dQ_q and the first left factor U (I - 2 S)
  BTRY(launch_bwd_gq(P->pm, P->qm[P->q], P->d_roff_m, P->d_qunits_m, P->nq_m, P->l, P->ub, P->sig, P->k, P->gm,
                     P->lbuf, kr, P->st));
  int blk = 1;
  for (int j = P->q; j >= 1; --j, blk += 2) {
    BTRYS(qr_back(P, P->qm[j], P->gm, P->rm[j], true, P->pm));                   // dY_j
    BTRY(launch_copy_block(P->pm, P->sum_m, P->lbuf, kr, blk * LP, P->st));
    BTRY(launch_copy_block(P->qn[j - 1], P->sum_n, P->rbuf, kr, blk * LP, P->st));
    BTRYS(to_operand(P, P->pm, true, 1));
    BTRYS(bpass(P, 1, 1, P->gn));                                                // dQt_j = A^T dY_j
    BTRYS(qr_back(P, P->qn[j - 1], P->gn, P->rn[j - 1], false, P->yn));          // dZ_j
    BTRY(launch_copy_block(P->yn, P->sum_n, P->rbuf, kr, (blk + 1) * LP, P->st));
    BTRY(launch_copy_block(P->qm[j - 1], P->sum_m, P->lbuf, kr, (blk + 1) * LP, P->st));
    BTRYS(to_operand(P, P->yn, false, 1));
    BTRYS(bpass(P, 0, 1, P->gm));                                                // dQ_{j-1} = A dZ_j
  }
  BTRYS(qr_back(P, P->qm[0], P->gm, P->rm[0], true, P->pm));                     // dY_0
  BTRY(launch_copy_block(P->pm, P->sum_m, P->lbuf, kr, blk * LP, P->st));
  BTRY(launch_copy_block(P->omega, P->sum_n, P->rbuf, kr, blk * LP, P->st));
  BTRY(launch_bwd_split(P->lbuf, P->sum_m * kr, P->lplanes, P->st));
  BTRY(launch_bwd_split(P->rbuf, P->sum_n * kr, P->rplanes, P->st));
  BTRY(launch_bwd_final(P->map_lp, P->map_rp, P->d_maps, P->d_units_f, P->nunits_f, P->sum_m, P->sum_n, kr,
                        P->d_gptr, P->d_m, P->d_n, P->d_roff_m, P->d_roff_n, P->num_sms, P->status, P->st));
  return RSVD_OK;
}

// Runs `body` once under stream capture and keeps the instantiated graph in *exec (one graph
// launch per call afterwards).  Falls back to direct launches where capture is not possible
// (the legacy default stream, or capture or instantiation refused).
template <class F>
rsvd_status_t run_captured(rsvd_batched_plan_t P, cudaGraphExec_t* exec, F body) {
  const bool can = P->use_graph && P->st != nullptr && P->st != cudaStreamLegacy &&
                   P->st != cudaStreamPerThread;
  if (!can) return body();
  if (!*exec) {
    if (cudaStreamBeginCapture(P->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return body();
    }
    const rsvd_status_t st = body();
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(P->st, &graph);
    if (st != RSVD_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (ce != cudaSuccess || !graph) {
      cudaGetLastError();
      return body();
    }
    const cudaError_t ie = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      cudaGetLastError();
      *exec = nullptr;
      return body();
    }
  }
  BTRY(cudaGraphLaunch(*exec, P->st));
  return RSVD_OK;
}

}  // namespace
}  // namespace rsvd

using namespace rsvd;

extern "C" {

rsvd_status_t rsvd_batched_plan_create(rsvd_batched_plan_t* plan, int32_t batch, const int64_t* m,
                                       const int64_t* n, const int64_t* lda, int32_t k, int32_t p,
                                       int32_t q, uint64_t seed, const rsvd_options_t* opt,
                                       void* stream) {
  if (!plan) return RSVD_ERR_INVALID_ARG;
  *plan = nullptr;
  if (batch < 1 || !m || !n || k < 1 || p < 0 || q < 0 || k + p > kBatchedLP) return RSVD_ERR_INVALID_ARG;
  rsvd_options_t o;
  if (opt) o = *opt; else rsvd_options_default(&o);
  if (o.orth_rounds != 2 && o.orth_rounds != 3) return RSVD_ERR_INVALID_ARG;
  if (o.precision != RSVD_BF16_TC || o.dtype_A != RSVD_BF16 || o.test_matrix != RSVD_GAUSSIAN ||
      o.single_pass || o.residual_passes || o.host_f32 || o.recompute)
    return RSVD_ERR_UNSUPPORTED;   // the batched path is the bf16 tensor-core Gaussian form
  const int l = k + p;
  for (int b = 0; b < batch; ++b) {
    const int64_t ld = lda ? lda[b] : round_up(n[b], 8);
    if (m[b] < l || n[b] < l || ld < n[b] || (ld % 8) != 0 || m[b] >= (1ll << 31) ||
        n[b] >= (1ll << 31))
      return RSVD_ERR_INVALID_ARG;
  }
  rsvd_batched_plan_t P = new (std::nothrow) rsvd_batched_plan_s();
  if (!P) return RSVD_ERR_ALLOC;
  P->nb = batch; P->k = k; P->p = p; P->q = q; P->l = l; P->seed = seed; P->opt = o;
  {
    const char* e = getenv("RSVD_NO_GRAPH");
    P->use_graph = !(e && e[0] && e[0] != '0');
  }
  P->st = static_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      prepare_batched() != cudaSuccess || prepare_batched_bwd() != cudaSuccess) {
    cudaGetLastError();
    delete P;
    return RSVD_ERR_CUDA;
  }
  P->m.assign(m, m + batch);
  P->n.assign(n, n + batch);
  P->max_m = *std::max_element(P->m.begin(), P->m.end());
  P->max_n = *std::max_element(P->n.begin(), P->n.end());
  P->lda.resize(batch);
  std::vector<int64_t> roff_m(batch + 1, 0), roff_n(batch + 1, 0), xoff_m(batch), xoff_n(batch);
  for (int b = 0; b < batch; ++b) {
    P->lda[b] = lda ? lda[b] : round_up(n[b], 8);
    roff_m[b + 1] = roff_m[b] + m[b];
    roff_n[b + 1] = roff_n[b] + n[b];
    xoff_m[b] = P->xm_total;
    xoff_n[b] = P->xn_total;
    P->xm_total += round_up(m[b], 8);
    P->xn_total += round_up(n[b], 8);
  }
  P->sum_m = roff_m[batch];
  P->sum_n = roff_n[batch];
  const std::vector<int2> u0 = make_units(P->m, P->n), u1 = make_units(P->n, P->m);
  P->nunits0 = (int)u0.size();
  P->nunits1 = (int)u1.size();
  std::vector<int> us_m, us_n;
  const std::vector<int2> qu_m = make_qr_units(P->m, &us_m), qu_n = make_qr_units(P->n, &us_n);
  P->nq_m = (int)qu_m.size();
  P->nq_n = (int)qu_n.size();
  P->h_maps.assign((size_t)2 * batch * 128, 0);
  P->a_bound.assign(batch, nullptr);
  const int64_t ldx = std::max(P->xm_total, P->xn_total);
  rsvd_status_t s;
  if ((s = upload(P, &P->d_roff_m, roff_m)) != RSVD_OK || (s = upload(P, &P->d_roff_n, roff_n)) != RSVD_OK ||
      (s = upload(P, &P->d_xoff_m, xoff_m)) != RSVD_OK || (s = upload(P, &P->d_xoff_n, xoff_n)) != RSVD_OK ||
      (s = upload(P, &P->d_m, P->m)) != RSVD_OK || (s = upload(P, &P->d_n, P->n)) != RSVD_OK ||
      (s = upload(P, &P->d_units0, u0)) != RSVD_OK || (s = upload(P, &P->d_units1, u1)) != RSVD_OK ||
      (s = upload(P, &P->d_qunits_m, qu_m)) != RSVD_OK || (s = upload(P, &P->d_qunits_n, qu_n)) != RSVD_OK ||
      (s = upload(P, &P->d_ustart_m, us_m)) != RSVD_OK || (s = upload(P, &P->d_ustart_n, us_n)) != RSVD_OK ||
      (s = balloc(P, &P->qpart, (size_t)std::max(P->nq_m, P->nq_n) * LP * LP)) != RSVD_OK ||
      (s = balloc(P, &P->d_maps, P->h_maps.size())) != RSVD_OK ||
      (s = balloc(P, &P->xbf, (size_t)2 * LP * ldx)) != RSVD_OK ||
      (s = balloc(P, &P->omega, (size_t)P->sum_n * LP)) != RSVD_OK ||
      (s = balloc(P, &P->ym, (size_t)P->sum_m * LP)) != RSVD_OK ||
      (s = balloc(P, &P->yn, (size_t)P->sum_n * LP)) != RSVD_OK ||
      (s = balloc(P, &P->qb, (size_t)P->sum_n * LP)) != RSVD_OK ||
      (s = balloc(P, &P->rb, (size_t)batch * LP * LP)) != RSVD_OK ||
      (s = balloc(P, &P->ub, (size_t)batch * LP * LP)) != RSVD_OK ||
      (s = balloc(P, &P->wb, (size_t)batch * LP * LP)) != RSVD_OK ||
      (s = balloc(P, &P->sig, (size_t)batch * LP)) != RSVD_OK ||
      (s = balloc(P, &P->status, 4)) != RSVD_OK) {
    bfree(P);
    return s;
  }
  P->kr = kBatchedLP * (2 * q + 2);
  {
    std::vector<int4> uf;
    const int ft = bwd_final_tile();
    for (int b = 0; b < batch; ++b)
      for (int64_t rt = 0; rt < cdiv(m[b], ft); ++rt)
        for (int64_t ct = 0; ct < cdiv(n[b], ft); ++ct) uf.push_back(make_int4(b, (int)rt, (int)ct, 0));
    P->nunits_f = (int)uf.size();
    if ((s = upload(P, &P->d_units_f, uf)) != RSVD_OK || (s = upload(P, &P->d_lda, P->lda)) != RSVD_OK ||
        (s = balloc(P, &P->lbuf, (size_t)P->sum_m * P->kr)) != RSVD_OK ||
        (s = balloc(P, &P->rbuf, (size_t)P->sum_n * P->kr)) != RSVD_OK ||
        (s = balloc(P, &P->lplanes, (size_t)3 * P->sum_m * P->kr)) != RSVD_OK ||
        (s = balloc(P, &P->rplanes, (size_t)3 * P->sum_n * P->kr)) != RSVD_OK ||
        (s = balloc(P, &P->gm, (size_t)P->sum_m * LP)) != RSVD_OK ||
        (s = balloc(P, &P->pm, (size_t)P->sum_m * LP)) != RSVD_OK ||
        (s = balloc(P, &P->gn, (size_t)P->sum_n * LP)) != RSVD_OK ||
        (s = balloc(P, &P->nmat, (size_t)batch * LP * LP)) != RSVD_OK ||
        (s = balloc(P, &P->rinv, (size_t)batch * LP * LP)) != RSVD_OK ||
        (s = balloc(P, &P->d_aptr, (size_t)batch)) != RSVD_OK ||
        (s = balloc(P, &P->d_gptr, (size_t)batch)) != RSVD_OK) {
      bfree(P);
      return s;
    }
  }
  P->qm.assign(q + 1, nullptr);
  P->rm.assign(q + 1, nullptr);
  P->qn.assign(q, nullptr);
  P->rn.assign(q, nullptr);
  for (int j = 0; j <= q; ++j)
    if ((s = balloc(P, &P->qm[j], (size_t)P->sum_m * LP)) != RSVD_OK ||
        (s = balloc(P, &P->rm[j], (size_t)batch * LP * LP)) != RSVD_OK) {
      bfree(P);
      return s;
    }
  for (int j = 0; j < q; ++j)
    if ((s = balloc(P, &P->qn[j], (size_t)P->sum_n * LP)) != RSVD_OK ||
        (s = balloc(P, &P->rn[j], (size_t)batch * LP * LP)) != RSVD_OK) {
      bfree(P);
      return s;
    }
  if (tc_encode_2d(P->map_x_m, P->xbf, P->xm_total, LP, ldx, 64, LP) ||
      tc_encode_2d(P->map_x_n, P->xbf, P->xn_total, LP, ldx, 64, LP) ||
      tc_encode_2d(P->map_x_m2, P->xbf, P->xm_total, 2 * LP, ldx, 64, 2 * LP) ||
      tc_encode_2d(P->map_x_n2, P->xbf, P->xn_total, 2 * LP, ldx, 64, 2 * LP) ||
      tc_encode_2d(P->map_lp, P->lplanes, P->kr, 3 * P->sum_m, P->kr, 64, bwd_final_tile()) ||
      tc_encode_2d(P->map_rp, P->rplanes, P->kr, 3 * P->sum_n, P->kr, 64, bwd_final_tile()) ||
      cudaMemsetAsync(P->xbf, 0, sizeof(__nv_bfloat16) * 2 * LP * ldx, P->st) != cudaSuccess ||
      cudaMemsetAsync(P->status, 0, 4 * sizeof(uint32_t), P->st) != cudaSuccess) {
    cudaGetLastError();
    bfree(P);
    return RSVD_ERR_CUDA;
  }
  *plan = P;
  return RSVD_OK;
}

rsvd_status_t rsvd_batched_plan_destroy(rsvd_batched_plan_t P) {
  if (!P) return RSVD_OK;
  cudaStreamSynchronize(P->st);
  bfree(P);
  return RSVD_OK;
}

rsvd_status_t rsvd_batched_svd(rsvd_batched_plan_t P, const void* const* A, float* U, float* S, float* V) {
  if (!P || !A || !U || !S || !V) return RSVD_ERR_INVALID_ARG;
  // the tensor maps of the A_b are encoded and copied to the device outside the graph; the
  // graph (all kernels of the forward) is kept while the plan sees the same pointers
  BTRYS(bind_maps(P, A));
  if (P->opt.autotune && !P->tuned) BTRYS(autotune(P));   // before the graph is captured
  const std::vector<const void*> a(A, A + P->nb);
  if (P->g_fwd && !(a == P->g_fwd_a && U == P->g_u && S == P->g_s && V == P->g_v)) {
    cudaGraphExecDestroy(P->g_fwd);
    P->g_fwd = nullptr;
  }
  P->g_fwd_a = a;
  P->g_u = U; P->g_s = S; P->g_v = V;
  return run_captured(P, &P->g_fwd, [&] { return bforward(P, A, U, S, V); });
}

rsvd_status_t rsvd_batched_svd_backward(rsvd_batched_plan_t P, const void* const* A, float* const* gA) {
  if (!P || !A || !gA) return RSVD_ERR_INVALID_ARG;
  for (int b = 0; b < P->nb; ++b)
    if (!gA[b]) return RSVD_ERR_INVALID_ARG;
  BTRYS(bind_maps(P, A));
  // the pointer arrays the final kernel reads go to the device outside the graph too
  BTRY(cudaMemcpyAsync(P->d_aptr, A, sizeof(void*) * P->nb, cudaMemcpyHostToDevice, P->st));
  BTRY(cudaMemcpyAsync(P->d_gptr, gA, sizeof(float*) * P->nb, cudaMemcpyHostToDevice, P->st));
  const std::vector<const void*> a(A, A + P->nb);
  const std::vector<float*> g(gA, gA + P->nb);
  if (P->g_bwd && !(a == P->g_bwd_a && g == P->g_bwd_g)) {
    cudaGraphExecDestroy(P->g_bwd);
    P->g_bwd = nullptr;
  }
  P->g_bwd_a = a;
  P->g_bwd_g = g;
  return run_captured(P, &P->g_bwd, [&] { return bbackward(P, A, gA); });
}

rsvd_status_t rsvd_batched_tuning(rsvd_batched_plan_t P, int32_t* stages, int32_t* ctas,
                                  int32_t* tuned) {
  if (!P) return RSVD_ERR_INVALID_ARG;
  for (int c = 0; c < 4; ++c) {
    if (stages) stages[c] = P->cfg_stages[c];
    if (ctas) ctas[c] = P->cfg_ctas[c];
  }
  if (tuned) *tuned = P->tuned ? 1 : 0;
  return RSVD_OK;
}

rsvd_status_t rsvd_batched_sync(rsvd_batched_plan_t P, uint32_t* sweeps) {
  if (!P) return RSVD_ERR_INVALID_ARG;
  uint32_t w[2] = {0, 0};
  BTRY(cudaMemcpyAsync(w, P->status, sizeof(w), cudaMemcpyDeviceToHost, P->st));
  BTRY(cudaStreamSynchronize(P->st));
  if (sweeps) *sweeps = w[1];
  if (w[0] || w[1]) BTRY(cudaMemsetAsync(P->status, 0, 2 * sizeof(uint32_t), P->st));
  if (w[0] & ST_NONFINITE) return RSVD_ERR_NONFINITE;
  if (w[0] & ST_TIMEOUT) return RSVD_ERR_TIMEOUT;
  if (w[0] & ST_NUMERICAL) return RSVD_ERR_NUMERICAL;
  return RSVD_OK;
}

}  // extern "C"
