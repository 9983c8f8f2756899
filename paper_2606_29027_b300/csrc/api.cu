// C ABI of libslar.so (declared in include/slar.h): argument checks, allocation of the
// context, and the entry points that are thin orchestration of the kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "context.cuh"
#include "macro.cuh"

namespace slar {
namespace {
std::atomic<long long> g_launches{0};
}
int count_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return 0;
}
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace slar

using namespace slar;

namespace {

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * n);
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

slar_status validate(const slar_config* cfg, char* msg, size_t len) {
  if (!cfg) { snprintf(msg, len, "null config"); return SLAR_EINVAL; }
  if (!((cfg->dx == 1 && cfg->dv == 1) || (cfg->dx == 2 && cfg->dv == 2))) {
    snprintf(msg, len, "dx = dv in {1, 2} required"); return SLAR_EINVAL;
  }
  const int d = cfg->dx + cfg->dv;
  for (int m = 0; m < d; ++m) {
    if (cfg->N[m] < 4 || cfg->N[m] > SLAR_MAX_N) {
      snprintf(msg, len, "N[%d] = %d outside [4, %d]", m, cfg->N[m], SLAR_MAX_N); return SLAR_EINVAL;
    }
    if (!(cfg->hi[m] > cfg->lo[m])) { snprintf(msg, len, "empty box in dim %d", m); return SLAR_EINVAL; }
  }
  for (int m = 0; m < cfg->dx; ++m)
    if (!is_pow2(cfg->N[m])) {
      snprintf(msg, len, "spatial N[%d] = %d must be a power of two (FFT)", m, cfg->N[m]);
      return SLAR_EINVAL;
    }
  if (cfg->dv == 2 && cfg->N[2] != cfg->N[3]) {
    snprintf(msg, len, "velocity dimensions must have equal N"); return SLAR_EINVAL;
  }
  if (cfg->rank_cap < 1 || cfg->rank_cap > SLAR_MAX_RANK) {
    snprintf(msg, len, "rank_cap must be in [1, %d]", SLAR_MAX_RANK); return SLAR_EINVAL;
  }
  if (!(cfg->eps >= 0.0)) { snprintf(msg, len, "eps must be >= 0"); return SLAR_EINVAL; }
  if (cfg->precision != SLAR_FP64 && cfg->precision != SLAR_FP32 && cfg->precision != SLAR_FP32_BF16X3 &&
      cfg->precision != SLAR_FP32_BF16X6) {
    snprintf(msg, len, "unknown precision"); return SLAR_EINVAL;
  }
  if (cfg->flags & ~(SLAR_LOMAC | SLAR_FOOT_EULER | SLAR_PROFILE | SLAR_PROFILE_EVAL | SLAR_PRECOND | SLAR_LEARNED |
                     SLAR_NO_AUTOTUNE | SLAR_OWN_STREAM | SLAR_DIRK_ONLY)) {
    snprintf(msg, len, "unknown flag bits"); return SLAR_EINVAL;
  }
  if (cfg->interp_order != 0 && cfg->interp_order != 2 && cfg->interp_order != 4) {
    snprintf(msg, len, "interp_order must be 0, 2 or 4"); return SLAR_EINVAL;
  }
  if (cfg->interp_order == 4) {
    if (cfg->precision != SLAR_FP64) {
      snprintf(msg, len, "interp_order 4 needs SLAR_FP64 entries"); return SLAR_EINVAL;
    }
    for (int m = 0; m < d; ++m)
      if (cfg->N[m] < 5) { snprintf(msg, len, "interp_order 4 needs N >= 5"); return SLAR_EINVAL; }
  }
  if (cfg->krylov_restart < 1 || cfg->krylov_restart > 64) {
    snprintf(msg, len, "krylov_restart must be in [1, 64]"); return SLAR_EINVAL;
  }
  if (cfg->aca_block < 0 || cfg->aca_block > ACA_BMAX) {
    snprintf(msg, len, "aca_block must be in [0, %d]", ACA_BMAX); return SLAR_EINVAL;
  }
  return SLAR_OK;
}

void free_ctx(slar_ctx* c) {
  if (!c) return;
  auto F = [](void* p) { if (p) cudaFree(p); };
  for (int sl = 0; sl < NSLOT; ++sl) {
    for (int m = 0; m < 4; ++m) F(c->ht[sl].U[m]);
    F(c->ht[sl].B12); F(c->ht[sl].B34); F(c->ht[sl].Broot);
  }
  for (int m = 0; m < 4; ++m) { F(c->U32[m]); F(c->Qleaf[m]); F(c->Rleaf[m]); }
  F(c->B12_32); F(c->B34_32); F(c->Broot32); F(c->tc_b12); F(c->tc_b34); F(c->tc_scratch); F(c->tc_broot); F(c->Ik); F(c->Lt[0]); F(c->Lt[1]);
  F(c->dC); F(c->qv); F(c->dC32); F(c->qv32); F(c->E32); F(c->Uc); F(c->Uh1); F(c->Uh2);
  F(c->Ua); F(c->Va); F(c->rowbuf); F(c->usedr); F(c->usedc); F(c->pivI); F(c->pivJ);
  F(c->ast); F(c->aca_part); F(c->aca_dots);
  F(c->chk_rows); F(c->chk_idx); F(c->chk_R); F(c->chk_n2); F(c->chk_n2t);
  if (c->aca_graph_blk) cudaGraphExecDestroy(c->aca_graph_blk);
  if (c->ast_host) cudaFreeHost(c->ast_host);
  if (c->evp) cudaFree(c->evp);
  if (c->evp_host) cudaFreeHost(c->evp_host);
  if (c->aca_graph) cudaGraphExecDestroy(c->aca_graph);
  if (c->h_ranks) cudaFreeHost(c->h_ranks);
  if (c->scal_host) cudaFreeHost(c->scal_host);
  F(c->T1); F(c->T2); F(c->T3); F(c->Q12); F(c->Q34); F(c->Rn[0]); F(c->Rn[1]);
  F(c->sm1); F(c->sm2); F(c->sm3); F(c->sm4);
  for (int t = 0; t < 6; ++t) { F(c->G[t]); F(c->W[t]); F(c->S[t]); F(c->ework[t]); }
  F(c->Sw);
  F(c->gram_work); F(c->tau); F(c->norm2); F(c->d_ranks); F(c->d_info); F(c->d_eig); F(c->d_rank);
  F(c->E); F(c->E1); F(c->E2); F(c->E3); F(c->mom); F(c->lvec); F(c->spec); F(c->rho); F(c->Wdev);
  F(c->macro_ws); F(c->scal);
  if (c->spectral) { c->spectral->release(); delete c->spectral; }
  if (c->cap_s) cudaStreamDestroy(c->cap_s);
  if (c->own_s) { cudaStreamSynchronize(c->own_s); cudaStreamDestroy(c->own_s); }
  macro_free(c);
  for (int i = 0; i < kProfEvents; ++i)
    if (c->prof_ev[i]) cudaEventDestroy(c->prof_ev[i]);
  for (int i = 0; i < 2; ++i)
    if (c->tune_ev[i]) cudaEventDestroy(c->tune_ev[i]);
  for (int i = 0; i < kPhaseEvents; ++i)
    if (c->ph_ev[i]) cudaEventDestroy(c->ph_ev[i]);
  delete c;
}

}  // namespace

extern "C" {

slar_status slar_create(const slar_config* cfg, void* stream, slar_ctx** out) {
  if (!out) return SLAR_EINVAL;
  *out = nullptr;
  char msg[256];
  slar_status st = validate(cfg, msg, sizeof(msg));
  if (st != SLAR_OK) { fprintf(stderr, "slar_create: %s\n", msg); return st; }
  slar_ctx* c = new (std::nothrow) slar_ctx();
  if (!c) return SLAR_ENOMEM;
  c->cfg = *cfg;
  if (c->cfg.delta_floor <= 0.0) c->cfg.delta_floor = 1e-12;
  if (c->cfg.newton_max <= 0) c->cfg.newton_max = 20;
  if (c->cfg.krylov_max <= 0) c->cfg.krylov_max = 200;
  c->s = static_cast<cudaStream_t>(stream);
  if (cfg->flags & SLAR_OWN_STREAM) {
    if (cudaStreamCreateWithFlags(&c->own_s, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return SLAR_ECUDA;
    }
    c->s = c->own_s;
  }
  c->dx = cfg->dx;
  c->dv = cfg->dv;
  c->d = cfg->dx + cfg->dv;
  GridDesc& g = c->g;
  g.d = c->d; g.dx = c->dx; g.dv = c->dv;
  g.NX = 1; g.NV = 1;
  g.S = cfg->interp_order == 4 ? 5 : 3;
  for (int m = 0; m < 4; ++m) {
    g.N[m] = m < c->d ? cfg->N[m] : 1;
    g.lo[m] = m < c->d ? cfg->lo[m] : 0.0;
    g.h[m] = m < c->d ? (cfg->hi[m] - cfg->lo[m]) / cfg->N[m] : 1.0;
    g.lof[m] = (float)g.lo[m];
    g.hf[m] = (float)g.h[m];
    g.ih[m] = 1.0 / g.h[m];
    g.ihf[m] = (float)g.ih[m];
  }
  for (int m = 0; m < c->dx; ++m) g.NX *= g.N[m];
  for (int m = 0; m < c->dv; ++m) g.NV *= g.N[c->dx + m];
  c->NX = g.NX;
  c->NV = g.NV;
  c->M1 = g.NX;
  c->M2 = g.NV;
  c->kmax = std::min(cfg->rank_cap, std::min(c->M1, c->M2));
  c->n_mom = c->dv == 1 ? 5 : 9;
  const int R = SLAR_MAX_RANK;
  const int d = c->d;
  long long capB = (long long)R * R * R;
  if (d == 4) {
    capB = std::max(capB, (long long)c->kmax * g.N[0] * g.N[1]);
    capB = std::max(capB, (long long)c->kmax * g.N[2] * g.N[3]);
  } else {
    capB = std::max(capB, (long long)std::max(c->M1, c->M2) * R);
  }
  capB = std::max(capB, (long long)SLAR_MAX_N * R * 9);
  c->capB = capB;
#define A(p, n) do { cudaError_t e_ = dalloc(&(p), (size_t)(n)); if (e_ != cudaSuccess) { free_ctx(c); return SLAR_ENOMEM; } } while (0)
  for (int sl = 0; sl < NSLOT; ++sl) {
    for (int m = 0; m < d; ++m) A(c->ht[sl].U[m], (size_t)g.N[m] * R);
    if (d == 4) { A(c->ht[sl].B12, (size_t)R * R * R); A(c->ht[sl].B34, (size_t)R * R * R); }
    A(c->ht[sl].Broot, (size_t)R * R);
  }
  for (int m = 0; m < d; ++m) {
    A(c->U32[m], (size_t)g.N[m] * R);
    A(c->Qleaf[m], (size_t)g.N[m] * R);
    A(c->Rleaf[m], (size_t)R * R);
  }
  if (d == 4) { A(c->B12_32, (size_t)R * R * R); A(c->B34_32, (size_t)R * R * R); }
  A(c->Broot32, (size_t)R * R);
  if (tc_pieces(c) > 0) {
    // prologue scratch for the largest launch: a block of ACA_BMAX fibres (or the check
    // rows) of the longer matricisation side, whole 128-entry tiles
    const long long cap = ((long long)ACA_BMAX * std::max(c->M1, c->M2) + 127) / 128 * 128;
    if (cudaMalloc(&c->tc_b12, (size_t)tc_split_bytes(tc_pieces(c))) != cudaSuccess ||
        cudaMalloc(&c->tc_b34, (size_t)tc_split_bytes(tc_pieces(c))) != cudaSuccess ||
        cudaMalloc(&c->tc_scratch, (size_t)tc_scratch_bytes(cap)) != cudaSuccess ||
        cudaMalloc(&c->tc_broot, (size_t)64 * 64 * 2 * 3) != cudaSuccess) {
      free_ctx(c);
      return SLAR_ENOMEM;
    }
    c->tc_sc = tc_scratch_view(c->tc_scratch, cap);
  }
  A(c->Ik, (size_t)R * R);
  if (d == 2) { A(c->Lt[0], (size_t)c->M1 * c->kmax); A(c->Lt[1], (size_t)c->M2 * c->kmax); }
  A(c->dC, (size_t)(c->dv + 2) * c->NX);
  A(c->qv, (size_t)3 * c->dv * g.N[c->dx]);
  if (cfg->precision != SLAR_FP64) {
    A(c->dC32, (size_t)(c->dv + 2) * c->NX);
    A(c->qv32, (size_t)3 * c->dv * g.N[c->dx]);
    A(c->E32, (size_t)c->dx * c->NX);
  }
  A(c->Uc, (size_t)(c->dv + 2) * c->NX);
  A(c->Uh1, (size_t)(c->dv + 2) * c->NX);
  A(c->Uh2, (size_t)(c->dv + 2) * c->NX);
  A(c->Ua, (size_t)c->M1 * c->kmax);
  A(c->Va, (size_t)c->M2 * c->kmax);
  A(c->rowbuf, (size_t)ACA_BMAX * c->M2);
  A(c->usedr, (size_t)c->M1);
  A(c->usedc, (size_t)c->M2);
  A(c->pivI, (size_t)c->kmax);
  A(c->pivJ, (size_t)c->kmax);
  A(c->ast, 1);
  const int nbu = (c->M1 + 255) / 256, nbv = (c->M2 + 255) / 256;
  // partial sums of the cross-approximation post kernels: per block of rows, R + 1 slots
  // (one-fibre steps) or ACA_BMAX (R + ACA_BMAX) + 1 (block steps)
  A(c->aca_part, (size_t)(nbu + nbv) * (ACA_BMAX * (R + ACA_BMAX) + 1));
  // check rows of the cross-approximation stop test: distinct floor(frac(c g) M1),
  // g = (sqrt 5 - 1)/2, c = 1, 2, ...; at most 8
  std::vector<int> rows;
  {
    const double gold = (std::sqrt(5.0) - 1.0) / 2.0;
    for (int q = 1; (int)rows.size() < std::min(8, c->M1) && q <= 64 * 8 + c->M1; ++q) {
      const int i = (int)std::floor(std::fmod(q * gold, 1.0) * c->M1);
      if (std::find(rows.begin(), rows.end(), i) == rows.end()) rows.push_back(i);
    }
  }
  c->n_chk = (int)rows.size();
  A(c->chk_rows, (size_t)c->n_chk);
  A(c->chk_idx, (size_t)c->n_chk * c->M2 * d);
  A(c->chk_R, (size_t)c->n_chk * c->M2);
  A(c->chk_n2, (size_t)c->n_chk);
  A(c->chk_n2t, (size_t)c->n_chk * ACA_BMAX);
  A(c->T1, (size_t)capB); A(c->T2, (size_t)capB); A(c->T3, (size_t)capB);
  A(c->Q12, (size_t)capB); A(c->Q34, (size_t)capB);
  A(c->Rn[0], (size_t)R * R); A(c->Rn[1], (size_t)R * R);
  A(c->sm1, (size_t)R * R); A(c->sm2, (size_t)R * R); A(c->sm3, (size_t)R * R); A(c->sm4, (size_t)R * R);
  A(c->Sw, (size_t)4 * SLAR_MAX_N * SLAR_MAX_N);
  for (int t = 0; t < 6; ++t) {
    A(c->G[t], (size_t)SLAR_MAX_N * SLAR_MAX_N);
    A(c->W[t], (size_t)SLAR_MAX_N);
    A(c->S[t], (size_t)SLAR_MAX_N * SLAR_MAX_N);
    A(c->ework[t], (size_t)2 * (SLAR_MAX_N + 1) * (SLAR_MAX_N + 1));
  }
  const long long gram_rows = std::max((long long)std::max(c->M1, c->M2), capB / 1);
  c->gram_work_blocks = (int)((std::min(gram_rows, (long long)SLAR_MAX_N * SLAR_MAX_N) + 63) / 64);
  A(c->gram_work, (size_t)c->gram_work_blocks * R * R);
  A(c->tau, (size_t)R);
  A(c->norm2, 4);
  A(c->d_ranks, 8);
  A(c->d_info, 2);
  A(c->d_eig, 6);
  A(c->d_rank, 6);
  A(c->E, (size_t)c->dx * c->NX); A(c->E1, (size_t)c->dx * c->NX);
  A(c->E2, (size_t)c->dx * c->NX); A(c->E3, (size_t)c->dx * c->NX);
  A(c->mom, (size_t)c->n_mom * c->NX);
  A(c->lvec, (size_t)2 * 4 * 64 + 9 * 64 + 9 * 64 * 64 + 9 * 64);
  c->spec_len = (long long)2 * 24 * c->NX;
  A(c->spec, (size_t)c->spec_len);
  A(c->rho, (size_t)c->NX);
  A(c->Wdev, 8);
#undef A
  if (cudaMalloc(&c->evp, 256) != cudaSuccess || cudaMallocHost(&c->evp_host, 256) != cudaSuccess ||
      cudaMallocHost(&c->ast_host, sizeof(AcaState)) != cudaSuccess ||
      cudaMallocHost(&c->h_ranks, sizeof(int) * 16) != cudaSuccess ||
      cudaMallocHost(&c->scal_host, sizeof(double) * 64) != cudaSuccess) {
    free_ctx(c);
    return SLAR_ENOMEM;
  }
  if (cudaMemset(c->ast, 0, sizeof(AcaState)) != cudaSuccess) { free_ctx(c); return SLAR_ECUDA; }
  if (sl_eval_init_attrs() != cudaSuccess || linalg_init_attrs() != cudaSuccess ||
      (c->tc_b12 && sl_eval_tc_init_attrs() != cudaSuccess)) {
    free_ctx(c);
    return SLAR_ECUDA;
  }
  {
    // index tuples of the check rows: row i (spatial multi-index) x every velocity column
    std::vector<int> tup((size_t)c->n_chk * c->M2 * d);
    for (int q = 0; q < c->n_chk; ++q)
      for (int j = 0; j < c->M2; ++j) {
        int* t = tup.data() + ((size_t)q * c->M2 + j) * d;
        const int i = rows[q];
        if (d == 2) { t[0] = i; t[1] = j; }
        else { t[0] = i / g.N[1]; t[1] = i % g.N[1]; t[2] = j / g.N[3]; t[3] = j % g.N[3]; }
      }
    if (cudaMemcpy(c->chk_rows, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->chk_idx, tup.data(), sizeof(int) * tup.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      free_ctx(c);
      return SLAR_ECUDA;
    }
  }
  if (cudaStreamCreateWithFlags(&c->cap_s, cudaStreamNonBlocking) != cudaSuccess) {
    free_ctx(c);
    return SLAR_ECUDA;
  }
  c->spectral = new (std::nothrow) Spectral();
  if (!c->spectral) { free_ctx(c); return SLAR_ENOMEM; }
  double L[2];
  for (int m = 0; m < c->dx; ++m) L[m] = cfg->hi[m] - cfg->lo[m];
  if (c->spectral->init(c->dx, cfg->N, L, c->s) != cudaSuccess) { free_ctx(c); return SLAR_ECUDA; }
  for (int i = 0; i < kProfEvents; ++i)
    if (cudaEventCreate(&c->prof_ev[i]) != cudaSuccess) { free_ctx(c); return SLAR_ECUDA; }
  for (int i = 0; i < kPhaseEvents; ++i)
    if (cudaEventCreate(&c->ph_ev[i]) != cudaSuccess) { free_ctx(c); return SLAR_ECUDA; }
  for (int i = 0; i < 2; ++i)
    if (cudaEventCreate(&c->tune_ev[i]) != cudaSuccess) { free_ctx(c); return SLAR_ECUDA; }
  const slar_status mst = macro_alloc(c);
  if (mst != SLAR_OK) { free_ctx(c); return mst; }
  *out = c;
  return SLAR_OK;
}

slar_status slar_destroy(slar_ctx* c) {
  if (!c) return SLAR_EINVAL;
  if (c->s) cudaStreamSynchronize(c->s); else cudaDeviceSynchronize();
  free_ctx(c);
  return SLAR_OK;
}

const char* slar_last_error(const slar_ctx* c) { return c ? c->err : "null context"; }

slar_status slar_launch_count(long long* out) {
  if (!out) return SLAR_EINVAL;
  *out = launch_count();
  return SLAR_OK;
}

slar_status slar_sizes(const slar_ctx* c, int* n_mom, int* nx) {
  if (!c) return SLAR_EINVAL;
  if (n_mom) *n_mom = c->n_mom;
  if (nx) *nx = c->NX;
  return SLAR_OK;
}

static int spare_slot(const slar_ctx* c, int a, int b = -1) {
  for (int s = 0; s < NSLOT; ++s)
    if (s != a && s != b) return s;
  return -1;
}

// U = (M0, M1, M2/2 + e_p(M0)) of the state, n_i optionally reset to mean(M0)
static slar_status conserved_of_state(slar_ctx* c, bool reset_ni) {
  CKS(compute_moments(c, c->cur, true, c->mom, c->dv + 2));
  if (reset_ni) {
    std::vector<double> m0(c->NX);
    CK(cudaMemcpyAsync(m0.data(), c->mom, sizeof(double) * c->NX, cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    double s = 0.0;
    for (double v : m0) s += v;
    c->n_i = s / c->NX;
  }
  CKS(field_from_M0(c, c->mom, c->E, nullptr, nullptr));
  return conserved_from_moments(c, c->mom, c->E, c->Uc);
}

slar_status init_ht(slar_ctx* c, int n_terms, const double* factors) {
  if (!c || !factors) return SLAR_EINVAL;
  if (n_terms < 1 || n_terms > SLAR_MAX_RANK)
    return set_error(c, SLAR_EINVAL, "n_terms must be in [1, 64]");
  const int d = c->d;
  for (int m = 0; m < d; ++m)
    if (n_terms > c->g.N[m]) return set_error(c, SLAR_EINVAL, "n_terms exceeds a grid size");
  int off[5] = {0, 0, 0, 0, 0};
  for (int m = 0; m < d; ++m) off[m + 1] = off[m] + c->g.N[m];
  const int tmp = spare_slot(c, c->cur);
  HTBuf& h = c->ht[tmp];
  const int T = n_terms;
  for (int m = 0; m < d; ++m) {
    const int N = c->g.N[m];
    std::vector<double> U((size_t)N * T);
    for (int t = 0; t < T; ++t)
      for (int i = 0; i < N; ++i) U[(size_t)i * T + t] = factors[(size_t)t * off[d] + off[m] + i];
    CK(cudaMemcpy(h.U[m], U.data(), sizeof(double) * U.size(), cudaMemcpyHostToDevice));
    h.r[m] = T;
  }
  std::vector<double> I((size_t)T * T, 0.0);
  for (int t = 0; t < T; ++t) I[(size_t)t * T + t] = 1.0;
  CK(cudaMemcpy(h.Broot, I.data(), sizeof(double) * I.size(), cudaMemcpyHostToDevice));
  if (d == 4) {
    std::vector<double> D((size_t)T * T * T, 0.0);
    for (int t = 0; t < T; ++t) D[((size_t)t * T + t) * T + t] = 1.0;
    CK(cudaMemcpy(h.B12, D.data(), sizeof(double) * D.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h.B34, D.data(), sizeof(double) * D.size(), cudaMemcpyHostToDevice));
    h.r[4] = h.r[5] = T;
  }
  h.valid = true;
  TruncIn in = trunc_in_of_slot(c, tmp);
  const int dst = spare_slot(c, tmp);
  const long long capped0 = c->rank_capped;
  CKS(truncate_into(c, in, c->cfg.eps, c->cfg.rank_cap, dst));
  h.valid = false;
  c->cur = dst;
  c->has_corr = 0;
  c->step = 0;
  c->dt_hist[0] = c->dt_hist[1] = 0.0;
  c->pc_age = -1;
  c->pc_off = 0;
  CKS(conserved_of_state(c, true));
  c->has_U = true;
  CK(cudaStreamSynchronize(c->s));
  if (c->rank_capped != capped0) return set_error(c, SLAR_ERANK, "rank cap reached with eps unmet (result valid)");
  return SLAR_OK;
}

slar_status ht_truncate(slar_ctx* c, double eps, int cap) {
  if (!c) return SLAR_EINVAL;
  if (!(eps >= 0.0) || cap < 1 || cap > SLAR_MAX_RANK) return set_error(c, SLAR_EINVAL, "bad eps or cap");
  if (!c->ht[c->cur].valid) return set_error(c, SLAR_EINVAL, "no HT state");
  const int dst = spare_slot(c, c->cur);
  const long long capped0 = c->rank_capped;
  CKS(truncate_into(c, trunc_in_of_slot(c, c->cur), eps, cap, dst));
  c->ht[c->cur].valid = false;
  c->cur = dst;
  CK(cudaStreamSynchronize(c->s));
  if (c->rank_capped != capped0) return set_error(c, SLAR_ERANK, "rank cap reached with eps unmet (result valid)");
  return SLAR_OK;
}

slar_status ht_eval(slar_ctx* c, long long n, const int* idx, double* out) {
  if (!c || n < 0 || (n > 0 && (!idx || !out))) return SLAR_EINVAL;
  EvalArgs a{};
  a.mode = EVAL_TUPLES;
  a.n = n;
  a.idx = idx;
  a.out = out;
  CKS(refresh_f32_fields(c, nullptr, true));
  return eval_entries(c, c->cur, true, a, 1);
}

slar_status sl_eval(slar_ctx* c, double tau, const double* E, long long n, const int* idx, double* out) {
  if (!c || n < 0 || !E || (n > 0 && (!idx || !out))) return SLAR_EINVAL;
  EvalArgs a{};
  a.mode = EVAL_TUPLES;
  a.n = n;
  a.idx = idx;
  a.out = out;
  a.tau = tau;
  a.E = E;
  a.foot_euler = (c->cfg.flags & SLAR_FOOT_EULER) ? 1 : 0;
  CKS(refresh_f32_fields(c, E, true));
  return eval_entries(c, c->cur, true, a, 0);
}

slar_status slar_advect(slar_ctx* c, double tau, const double* E, int* aca_rank, long long* entries) {
  if (!c || !E) return SLAR_EINVAL;
  const int dst = spare_slot(c, c->cur);
  const long long capped0 = c->rank_capped;
  CKS(slar_call(c, c->cur, true, tau, E, dst, aca_rank, entries));
  c->ht[c->cur].valid = false;
  c->cur = dst;
  c->has_corr = 0;
  if (c->rank_capped != capped0) return set_error(c, SLAR_ERANK, "rank cap reached with eps unmet (result valid)");
  return SLAR_OK;
}

slar_status slar_set_pivot_replay(slar_ctx* c, int n_calls, int kmax, const int* pivots) {
  if (!c || n_calls < 0 || (n_calls > 0 && (!pivots || kmax < 1))) return SLAR_EINVAL;
  c->replay.assign(pivots, pivots + (size_t)n_calls * kmax * 2);
  c->replay_calls = n_calls;
  c->replay_kmax = kmax;
  c->replay_pos = 0;
  return SLAR_OK;
}

slar_status moments(slar_ctx* c, unsigned mask, double* out) {
  if (!c || !out) return SLAR_EINVAL;
  if (mask & ~(unsigned)SLAR_MOM_ALL) return set_error(c, SLAR_EINVAL, "unknown moment mask bits");
  if (mask == 0) mask = SLAR_MOM_ALL;
  // rows of the full table in order: M0 | M1 (dv) | M2 | flux moments (n_mom - dv - 2)
  const int dv = c->dv;
  std::vector<int> rows;
  if (mask & SLAR_MOM_M0) rows.push_back(0);
  if (mask & SLAR_MOM_M1)
    for (int a = 0; a < dv; ++a) rows.push_back(1 + a);
  if (mask & SLAR_MOM_M2) rows.push_back(1 + dv);
  if (mask & SLAR_MOM_FLUX)
    for (int q = dv + 2; q < c->n_mom; ++q) rows.push_back(q);
  bool prefix = true;
  for (size_t i = 0; i < rows.size(); ++i) prefix = prefix && rows[i] == (int)i;
  if (prefix) return compute_moments(c, c->cur, true, out, (int)rows.size());
  CKS(compute_moments(c, c->cur, true, c->mom, rows.back() + 1));
  for (size_t i = 0; i < rows.size(); ++i)
    CK(cudaMemcpyAsync(out + (size_t)i * c->NX, c->mom + (size_t)rows[i] * c->NX, sizeof(double) * c->NX,
                       cudaMemcpyDeviceToDevice, c->s));
  return SLAR_OK;
}

slar_status poisson_field(slar_ctx* c, const double* rho, double* E, double* phi, double* energy) {
  if (!c || !rho || !E) return SLAR_EINVAL;
  CKS(poisson_dev(c, rho, E, phi, energy ? c->Wdev : nullptr));
  if (energy) {
    CK(cudaMemcpyAsync(c->scal_host, c->Wdev, sizeof(double), cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    *energy = c->scal_host[0];
  }
  return SLAR_OK;
}

slar_status ht_export(slar_ctx* c, slar_ht_view* v) {
  if (!c || !v) return SLAR_EINVAL;
  const HTBuf& h = c->ht[c->cur];
  if (!h.valid) return set_error(c, SLAR_EINVAL, "no HT state");
  v->d = c->d;
  for (int m = 0; m < 4; ++m) v->N[m] = m < c->d ? c->g.N[m] : 0;
  for (int i = 0; i < 6; ++i) v->rank[i] = h.r[i];
  v->has_corr = c->has_corr;
  bool any_null = !v->Broot;
  for (int m = 0; m < c->d; ++m) any_null |= !v->U[m];
  if (c->d == 4) any_null |= (!v->B12 || !v->B34);
  if (any_null) return SLAR_OK;
  CK(cudaStreamSynchronize(c->s));
  for (int m = 0; m < c->d; ++m)
    CK(cudaMemcpy(v->U[m], h.U[m], sizeof(double) * c->g.N[m] * h.r[m], cudaMemcpyDeviceToHost));
  if (c->d == 4) {
    CK(cudaMemcpy(v->B12, h.B12, sizeof(double) * h.r[4] * h.r[0] * h.r[1], cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(v->B34, h.B34, sizeof(double) * h.r[5] * h.r[2] * h.r[3], cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(v->Broot, h.Broot, sizeof(double) * h.r[4] * h.r[5], cudaMemcpyDeviceToHost));
  } else {
    CK(cudaMemcpy(v->Broot, h.Broot, sizeof(double) * h.r[0] * h.r[1], cudaMemcpyDeviceToHost));
  }
  if (c->has_corr && v->dC && v->qv) {
    CK(cudaMemcpy(v->dC, c->dC, sizeof(double) * (c->dv + 2) * c->NX, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(v->qv, c->qv, sizeof(double) * 3 * c->dv * c->g.N[c->dx], cudaMemcpyDeviceToHost));
  }
  return SLAR_OK;
}

slar_status ht_import(slar_ctx* c, const slar_ht_view* v) {
  if (!c || !v) return SLAR_EINVAL;
  if (v->d != c->d) return set_error(c, SLAR_EINVAL, "dimension mismatch");
  for (int m = 0; m < c->d; ++m) {
    if (v->N[m] != c->g.N[m]) return set_error(c, SLAR_EINVAL, "grid mismatch");
    if (v->rank[m] < 1 || v->rank[m] > SLAR_MAX_RANK || !v->U[m])
      return set_error(c, SLAR_EINVAL, "bad leaf rank or pointer");
  }
  if (c->d == 4)
    for (int i = 4; i < 6; ++i)
      if (v->rank[i] < 1 || v->rank[i] > SLAR_MAX_RANK)
        return set_error(c, SLAR_EINVAL, "bad node rank");
  if (!v->Broot || (c->d == 4 && (!v->B12 || !v->B34))) return set_error(c, SLAR_EINVAL, "null factor");
  const int dst = spare_slot(c, c->cur);
  HTBuf& h = c->ht[dst];
  for (int m = 0; m < c->d; ++m) {
    h.r[m] = v->rank[m];
    CK(cudaMemcpy(h.U[m], v->U[m], sizeof(double) * c->g.N[m] * h.r[m], cudaMemcpyHostToDevice));
  }
  if (c->d == 4) {
    h.r[4] = v->rank[4];
    h.r[5] = v->rank[5];
    CK(cudaMemcpy(h.B12, v->B12, sizeof(double) * h.r[4] * h.r[0] * h.r[1], cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h.B34, v->B34, sizeof(double) * h.r[5] * h.r[2] * h.r[3], cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h.Broot, v->Broot, sizeof(double) * h.r[4] * h.r[5], cudaMemcpyHostToDevice));
  } else {
    h.r[4] = h.r[5] = 0;
    CK(cudaMemcpy(h.Broot, v->Broot, sizeof(double) * h.r[0] * h.r[1], cudaMemcpyHostToDevice));
  }
  h.valid = true;
  c->ht[c->cur].valid = false;
  c->cur = dst;
  if (c->f32_slot == dst) c->f32_slot = -1;
  c->has_corr = 0;
  if (v->has_corr) {
    if (!v->dC || !v->qv) return set_error(c, SLAR_EINVAL, "correction arrays missing");
    CK(cudaMemcpy(c->dC, v->dC, sizeof(double) * (c->dv + 2) * c->NX, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->qv, v->qv, sizeof(double) * 3 * c->dv * c->g.N[c->dx], cudaMemcpyHostToDevice));
    c->has_corr = 1;
  }
  return SLAR_OK;
}

slar_status slar_get_conserved(slar_ctx* c, double* U, double* n_i) {
  if (!c) return SLAR_EINVAL;
  if (U) CK(cudaMemcpyAsync(U, c->Uc, sizeof(double) * (c->dv + 2) * c->NX, cudaMemcpyDeviceToDevice, c->s));
  if (n_i) *n_i = c->n_i;
  return SLAR_OK;
}

slar_status slar_set_conserved(slar_ctx* c, const double* U, double n_i) {
  if (!c || !U) return SLAR_EINVAL;
  CK(cudaMemcpyAsync(c->Uc, U, sizeof(double) * (c->dv + 2) * c->NX, cudaMemcpyDeviceToDevice, c->s));
  c->n_i = n_i;
  c->has_U = true;
  return SLAR_OK;
}

slar_status lomac_correct(slar_ctx* c, const double* U_target) {
  if (!c || !U_target) return SLAR_EINVAL;
  if (c->has_corr) return set_error(c, SLAR_EINVAL, "state already carries a correction");
  return lomac_apply(c, U_target);
}

slar_status slar_attach_net(slar_ctx* c, slar_net* net) {
  if (!c) return SLAR_EINVAL;
  if (net) {
    const int n1 = c->dx == 2 ? c->g.N[1] : 1;
    if (net_m(net) != c->dv + 2 || net_n0(net) != c->g.N[0] || net_n1(net) != n1)
      return set_error(c, SLAR_EINVAL, "network does not match the context's grid");
  }
  c->net = net;
  return SLAR_OK;
}

slar_status slar_set_record(slar_ctx* c, float* dst, int n_probes, unsigned long long seed) {
  if (!c || (dst && (n_probes < 1 || n_probes > 64))) return SLAR_EINVAL;
  c->rec_dst = dst;
  c->rec_S = n_probes;
  c->rec_seed = seed;
  return SLAR_OK;
}

slar_status slar_ensemble_step(slar_ctx** ctxs, int n, const double* dts, int threads, slar_stats* stats) {
  if (!ctxs || !dts || n < 1) return SLAR_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return SLAR_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i] || (n > 1 && ctxs[j]->s == ctxs[i]->s)) return SLAR_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SLAR_ECUDA;
  std::vector<slar_status> st(n, SLAR_OK);
  std::atomic<int> next{0};
  auto worker = [&]() {
    cudaSetDevice(dev);
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= n) break;
      st[i] = sl_step(ctxs[i], dts[i], stats ? &stats[i] : nullptr);
    }
  };
  const int nt = std::max(1, std::min(threads, n));
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  for (int i = 0; i < n; ++i)
    if (st[i] != SLAR_OK) return st[i];
  return SLAR_OK;
}

// ---------------- checkpoint / restore ----------------
namespace {

constexpr char kCkptMagic[8] = {'S', 'L', 'A', 'R', 'C', 'K', 'P', 'T'};
constexpr int kCkptVersion = 2;

// Fixed-size header of a checkpoint file (host byte order); the arrays follow in the order
// written by slar_checkpoint.
struct CkptHeader {
  char magic[8];
  int version;
  int d, dx, dv;
  int N[4];
  double lo[4], hi[4];
  int precision;
  int step, has_U, has_corr;
  int rank[6];
  int Sn[6];
  double n_i;
  long long net_np;   // parameters of the attached network saved (0: none)
  double dt_hist[2];  // sizes of the previous two steps (variable-step BDF3)
};

struct File {
  FILE* f = nullptr;
  ~File() { if (f) fclose(f); }
};

bool wr(FILE* f, const void* p, size_t bytes) { return fwrite(p, 1, bytes, f) == bytes; }
bool rd(FILE* f, void* p, size_t bytes) { return fread(p, 1, bytes, f) == bytes; }

// device FP64 array <-> file through a host buffer
slar_status dev_to_file(slar_ctx* c, FILE* f, const double* d, size_t n) {
  std::vector<double> h(n);
  if (n) CK(cudaMemcpy(h.data(), d, sizeof(double) * n, cudaMemcpyDeviceToHost));
  if (!wr(f, h.data(), sizeof(double) * n)) return set_error(c, SLAR_EINVAL, "checkpoint: write failed");
  return SLAR_OK;
}

slar_status file_to_dev(slar_ctx* c, FILE* f, double* d, size_t n) {
  std::vector<double> h(n);
  if (!rd(f, h.data(), sizeof(double) * n)) return set_error(c, SLAR_EINVAL, "restore: file truncated");
  if (n) CK(cudaMemcpy(d, h.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
  return SLAR_OK;
}

}  // namespace

slar_status slar_checkpoint(slar_ctx* c, const char* path) {
  if (!c || !path) return SLAR_EINVAL;
  const HTBuf& h = c->ht[c->cur];
  if (!h.valid || !c->has_U) return set_error(c, SLAR_EINVAL, "checkpoint: no state (call init_ht first)");
  CK(cudaStreamSynchronize(c->s));
  CkptHeader hd{};
  std::memcpy(hd.magic, kCkptMagic, 8);
  hd.version = kCkptVersion;
  hd.d = c->d; hd.dx = c->dx; hd.dv = c->dv;
  for (int m = 0; m < 4; ++m) { hd.N[m] = c->cfg.N[m]; hd.lo[m] = c->cfg.lo[m]; hd.hi[m] = c->cfg.hi[m]; }
  hd.precision = c->cfg.precision;
  hd.step = c->step; hd.has_U = c->has_U ? 1 : 0; hd.has_corr = c->has_corr;
  for (int i = 0; i < 6; ++i) { hd.rank[i] = h.r[i]; hd.Sn[i] = c->Sn[i]; }
  hd.n_i = c->n_i;
  hd.net_np = c->net ? net_np(c->net) : 0;
  hd.dt_hist[0] = c->dt_hist[0];
  hd.dt_hist[1] = c->dt_hist[1];
  File F;
  F.f = fopen(path, "wb");
  if (!F.f) return set_error(c, SLAR_EINVAL, "checkpoint: cannot open the file for writing");
  if (!wr(F.f, &hd, sizeof(hd))) return set_error(c, SLAR_EINVAL, "checkpoint: write failed");
  for (int m = 0; m < c->d; ++m) CKS(dev_to_file(c, F.f, h.U[m], (size_t)c->g.N[m] * h.r[m]));
  if (c->d == 4) {
    CKS(dev_to_file(c, F.f, h.B12, (size_t)h.r[4] * h.r[0] * h.r[1]));
    CKS(dev_to_file(c, F.f, h.B34, (size_t)h.r[5] * h.r[2] * h.r[3]));
    CKS(dev_to_file(c, F.f, h.Broot, (size_t)h.r[4] * h.r[5]));
  } else {
    CKS(dev_to_file(c, F.f, h.Broot, (size_t)h.r[0] * h.r[1]));
  }
  const size_t nU = (size_t)(c->dv + 2) * c->NX;
  if (c->has_corr) {
    CKS(dev_to_file(c, F.f, c->dC, nU));
    CKS(dev_to_file(c, F.f, c->qv, (size_t)3 * c->dv * c->g.N[c->dx]));
  }
  CKS(dev_to_file(c, F.f, c->Uc, nU));
  CKS(dev_to_file(c, F.f, c->Uh1, nU));
  CKS(dev_to_file(c, F.f, c->Uh2, nU));
  for (int t = 0; t < 6; ++t)
    if (c->Sn[t] > 0) CKS(dev_to_file(c, F.f, c->S[t], (size_t)c->Sn[t] * c->Sn[t]));
  if (hd.net_np > 0) {
    std::vector<float> th((size_t)hd.net_np);
    CKS(slar_net_get_params(c->net, th.data(), hd.net_np));
    if (!wr(F.f, th.data(), sizeof(float) * th.size())) return set_error(c, SLAR_EINVAL, "checkpoint: write failed");
  }
  if (fflush(F.f) != 0) return set_error(c, SLAR_EINVAL, "checkpoint: write failed");
  return SLAR_OK;
}

slar_status slar_restore(slar_ctx* c, const char* path) {
  if (!c || !path) return SLAR_EINVAL;
  File F;
  F.f = fopen(path, "rb");
  if (!F.f) return set_error(c, SLAR_EINVAL, "restore: cannot open the file");
  CkptHeader hd{};
  if (!rd(F.f, &hd, sizeof(hd)) || std::memcmp(hd.magic, kCkptMagic, 8) != 0 || hd.version != kCkptVersion)
    return set_error(c, SLAR_EINVAL, "restore: not a checkpoint of this library version");
  // the saved state is FP64 whatever the writer's entry precision, so a run may resume in
  // another precision; the grid and the box must be the same
  bool same = hd.d == c->d && hd.dx == c->dx && hd.dv == c->dv;
  for (int m = 0; m < 4; ++m)
    same = same && hd.N[m] == c->cfg.N[m] && hd.lo[m] == c->cfg.lo[m] && hd.hi[m] == c->cfg.hi[m];
  if (!same) return set_error(c, SLAR_EINVAL, "restore: grid or box differ from the context's");
  for (int i = 0; i < (c->d == 4 ? 6 : 2); ++i)
    if (hd.rank[i] < 1 || hd.rank[i] > SLAR_MAX_RANK) return set_error(c, SLAR_EINVAL, "restore: bad rank");
  for (int t = 0; t < 6; ++t)
    if (hd.Sn[t] < 0 || hd.Sn[t] > SLAR_MAX_N) return set_error(c, SLAR_EINVAL, "restore: bad basis order");
  if (hd.step < 0 || hd.has_U != 1 || (hd.has_corr != 0 && hd.has_corr != 1) || hd.net_np < 0 ||
      !(hd.dt_hist[0] >= 0.0) || !(hd.dt_hist[1] >= 0.0) || (hd.step >= 2 && !(hd.dt_hist[1] > 0.0)))
    return set_error(c, SLAR_EINVAL, "restore: bad header");
  CK(cudaStreamSynchronize(c->s));
  const int dst = spare_slot(c, c->cur);
  HTBuf& h = c->ht[dst];
  for (int i = 0; i < 6; ++i) h.r[i] = hd.rank[i];
  if (c->d == 2) h.r[2] = h.r[3] = h.r[4] = h.r[5] = 0;
  for (int m = 0; m < c->d; ++m) CKS(file_to_dev(c, F.f, h.U[m], (size_t)c->g.N[m] * h.r[m]));
  if (c->d == 4) {
    CKS(file_to_dev(c, F.f, h.B12, (size_t)h.r[4] * h.r[0] * h.r[1]));
    CKS(file_to_dev(c, F.f, h.B34, (size_t)h.r[5] * h.r[2] * h.r[3]));
    CKS(file_to_dev(c, F.f, h.Broot, (size_t)h.r[4] * h.r[5]));
  } else {
    CKS(file_to_dev(c, F.f, h.Broot, (size_t)h.r[0] * h.r[1]));
  }
  const size_t nU = (size_t)(c->dv + 2) * c->NX;
  if (hd.has_corr) {
    CKS(file_to_dev(c, F.f, c->dC, nU));
    CKS(file_to_dev(c, F.f, c->qv, (size_t)3 * c->dv * c->g.N[c->dx]));
  }
  CKS(file_to_dev(c, F.f, c->Uc, nU));
  CKS(file_to_dev(c, F.f, c->Uh1, nU));
  CKS(file_to_dev(c, F.f, c->Uh2, nU));
  for (int t = 0; t < 6; ++t)
    if (hd.Sn[t] > 0) CKS(file_to_dev(c, F.f, c->S[t], (size_t)hd.Sn[t] * hd.Sn[t]));
  if (hd.net_np > 0) {
    std::vector<float> th((size_t)hd.net_np);
    if (!rd(F.f, th.data(), sizeof(float) * th.size())) return set_error(c, SLAR_EINVAL, "restore: file truncated");
    if (c->net && net_np(c->net) == hd.net_np) CKS(slar_net_set_params(c->net, th.data(), hd.net_np));
  }
  h.valid = true;
  if (dst != c->cur) c->ht[c->cur].valid = false;
  c->cur = dst;
  if (c->f32_slot == dst) c->f32_slot = -1;
  c->has_corr = hd.has_corr;
  c->has_U = true;
  c->n_i = hd.n_i;
  c->step = hd.step;
  c->dt_hist[0] = hd.dt_hist[0];
  c->dt_hist[1] = hd.dt_hist[1];
  for (int t = 0; t < 6; ++t) c->Sn[t] = hd.Sn[t];
  c->pc_age = -1;   // the preconditioner is not saved: the next BDF3 step probes it again
  c->pc_off = 0;
  return SLAR_OK;
}

slar_status slar_stream(const slar_ctx* c, void** stream) {
  if (!c || !stream) return SLAR_EINVAL;
  *stream = c->s;
  return SLAR_OK;
}

slar_status sl_step(slar_ctx* c, double dt, slar_stats* stats) {
  if (!c) return SLAR_EINVAL;
  if ((c->cfg.flags & SLAR_LEARNED) && !c->net)
    return set_error(c, SLAR_EINVAL, "SLAR_LEARNED needs a network (slar_attach_net)");
  if (!c->ht[c->cur].valid || !c->has_U) return set_error(c, SLAR_EINVAL, "call init_ht first");
  if (!(dt > 0.0)) return set_error(c, SLAR_EINVAL, "dt must be > 0");
  if ((c->cfg.flags & SLAR_LOMAC) && !(c->cfg.flags & SLAR_DIRK_ONLY) && c->step >= 2 &&
      dt > kBdf3RatioMax * c->dt_hist[0] * (1.0 + 1e-12))
    return set_error(c, SLAR_EINVAL, "step ratio above the variable-step BDF3 stability bound");
  return step_impl(c, dt, stats);
}

slar_status slar_cfl_dt(slar_ctx* c, double cfl, double dt_max, double* dt) {
  if (!c || !dt || !(cfl > 0.0) || !(dt_max > 0.0)) return SLAR_EINVAL;
  if (!c->ht[c->cur].valid || !c->has_U) return set_error(c, SLAR_EINVAL, "call init_ht first");
  return cfl_dt(c, cfl, dt_max, dt);
}

}  // extern "C"
