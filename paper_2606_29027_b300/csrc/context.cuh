// The opaque slar_ctx: configuration, device state and all workspaces (allocated once in
// slar_create, sized by the grid and the rank limit).
#pragma once

#include <vector>

#include "common.cuh"
#include "spectral.cuh"

namespace slar {

constexpr int kProfEvents = 2048;
constexpr int kPhaseEvents = 256;
enum { PH_ACA = 0, PH_TRUNC = 1, PH_FIELD = 2, PH_CLOSURE = 3, PH_NEWTON = 4, PH_DIAG = 5, PH_END = 6 };
// mark the start of a phase on the context stream (no-op unless SLAR_PROFILE)
void phase(slar_ctx* c, int tag);
struct MacroWS;

// One HT tensor on the device (capacity: ranks <= SLAR_MAX_RANK).
struct HTBuf {
  double* U[4] = {nullptr, nullptr, nullptr, nullptr};
  double* B12 = nullptr;
  double* B34 = nullptr;
  double* Broot = nullptr;
  int r[6] = {0, 0, 0, 0, 0, 0};  // leaf ranks, r12, r34
  bool valid = false;
};

constexpr int NSLOT = 4;

struct AcaState {
  int k;          // number of accepted cross terms = index of the running step
  int done;       // set when the cross approximation stops
  int stop_row;   // 1 if it stopped on a vanishing residual row (that row was sampled)
  int replay;     // pivots are replayed from pivI / pivJ
  double normA2;  // running ||A_k||_F^2 estimate
  double piv;     // current pivot value
  double nv2;     // ||v_k||^2
  double eps;     // stopping tolerance
  int tc_err;     // set by the tensor-core evaluator if an MMA completion wait ran out
  unsigned int post_ctr;  // block tickets of k_aca_post (reset by its last block)
  int cap_binds;  // the rank cap is below min(M1, M2) (reaching it leaves an error)
  int capped;     // stopped at the rank cap with the stop test unmet
  double piv0;    // |first pivot|: the scale of the negligible-row test
  int skip;       // the current row was negligible: no term this step
  int n_skip;     // negligible rows sampled in this call
  // block cross approximation
  int nrows;      // rows of the current block, at pivI[k .. k + nrows)
  int nact;       // pivots accepted in the current block (columns sampled)
  int rows_sampled;  // row and column fibres sampled by the block steps of this call
  int cols_sampled;
  int nsteps;        // block steps run in this call
};

constexpr int ACA_BMAX = 8;   // largest block of the block cross approximation

}  // namespace slar

struct slar_net;

struct slar_ctx {
  slar_config cfg;
  cudaStream_t s = nullptr;        // caller's stream: all work is ordered on it
  cudaStream_t cap_s = nullptr;    // internal stream used only to capture CUDA graphs
  cudaStream_t own_s = nullptr;    // private stream (SLAR_OWN_STREAM)
  slar::GridDesc g;
  int d = 0, dx = 0, dv = 0, NX = 0, NV = 0, M1 = 0, M2 = 0, kmax = 0, n_mom = 0;
  long long capB = 0;

  // HT slots (FP64 master); `cur` holds the state F^n, the others are RKEI stages.
  // The FP32 shadow mirrors slot `f32_slot` (-1 = stale).
  slar::HTBuf ht[slar::NSLOT];
  int cur = 0;
  int f32_slot = -1;
  float* U32[4] = {nullptr, nullptr, nullptr, nullptr};
  float* B12_32 = nullptr;
  float* B34_32 = nullptr;
  float* Broot32 = nullptr;
  void* tc_scratch = nullptr;   // the tensor-core evaluator's prologue scratch (tc_sc views it)
  slar::TcScratch tc_sc{};
  void* tc_broot = nullptr;  // the FP32 shadow's root matrix pre-split for the tensor cores
  void* tc_b12 = nullptr;   // BF16x3 pre-split transfer tensors of the FP32 shadow
  void* tc_b34 = nullptr;
  double* Ik = nullptr;     // identity (kmax x kmax)
  double* Lt[2] = {nullptr, nullptr};  // d = 2 cross factors as row-major leaves

  // separable LoMaC correction of the state
  int has_corr = 0;
  double* dC = nullptr;   // [dv+2][NX]
  double* qv = nullptr;   // [3][dv][Nv]
  float* dC32 = nullptr;  // FP32 copies of dC, qv and of the SLAR field (FP32 / BF16x3 paths)
  float* qv32 = nullptr;
  float* E32 = nullptr;   // [dx][NX]

  // macroscopic state
  double* Uc = nullptr;   // U^n       [dv+2][NX]
  double* Uh1 = nullptr;  // U^{n-1}
  double* Uh2 = nullptr;  // U^{n-2}
  double n_i = 1.0;
  int step = 0;
  bool has_U = false;
  double dt_hist[2] = {0.0, 0.0};   // sizes of the previous two steps (most recent first)

  // cross approximation
  double* Ua = nullptr;   // M1 x kmax column-major
  double* Va = nullptr;   // M2 x kmax
  double* rowbuf = nullptr;
  unsigned char* usedr = nullptr;
  unsigned char* usedc = nullptr;
  int* pivI = nullptr;
  int* pivJ = nullptr;
  slar::AcaState* ast = nullptr;
  slar::AcaState* ast_host = nullptr;  // pinned
  double* aca_part = nullptr;          // partial dot products
  double* aca_dots = nullptr;
  std::vector<int> replay;             // [calls][kmax][2]
  void* evp = nullptr;                 // device EvalParams of the running SLAR call
  void* evp_host = nullptr;            // pinned staging
  cudaGraphExec_t aca_graph = nullptr; // one cross-approximation step inside a WHILE node
  size_t aca_graph_smem = 0;
  long long aca_graph_nodes = 0;
  int replay_calls = 0, replay_kmax = 0, replay_pos = 0;
  // entry-evaluator tile (entries per CTA) chosen by the autotuner, and the tile the
  // cross-approximation graph was captured with
  int eval_tile = 32;
  int aca_graph_tile = 0;
  cudaEvent_t tune_ev[2] = {nullptr, nullptr};
  // check rows of the cross-approximation stop test
  int n_chk = 0;
  int* chk_rows = nullptr;     // [n_chk]
  int* chk_idx = nullptr;      // [n_chk * M2][d] index tuples of the check rows
  double* chk_R = nullptr;     // [n_chk][M2] residual rows
  double* chk_n2 = nullptr;    // [n_chk] their squared norms
  double* chk_n2t = nullptr;   // [n_chk][ACA_BMAX] the norms after each term of a block
  cudaGraphExec_t aca_graph_blk = nullptr;   // the block cross-approximation loop
  size_t aca_graph_blk_smem = 0;
  long long aca_graph_blk_nodes = 0;
  int aca_graph_blk_tile = 0;

  // truncation workspaces
  double* Qleaf[4] = {nullptr, nullptr, nullptr, nullptr};
  double* Rleaf[4] = {nullptr, nullptr, nullptr, nullptr};
  double* T1 = nullptr;
  double* T2 = nullptr;
  double* T3 = nullptr;
  double* Q12 = nullptr;
  double* Q34 = nullptr;
  double* Rn[2] = {nullptr, nullptr};
  double* sm1 = nullptr;  // small scratch matrices (64 x 64 each)
  double* sm2 = nullptr;
  double* sm3 = nullptr;
  double* sm4 = nullptr;
  double* G[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double* W[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double* S[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int Sn[6] = {0, 0, 0, 0, 0, 0};   // order of the eigenvector matrix kept in S[t] (warm start)
  double* Sw = nullptr;             // warm-start scratch (4 x 128 x 128)
  double* ework[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double* gram_work = nullptr;
  int gram_work_blocks = 0;
  double* tau = nullptr;
  double* norm2 = nullptr;
  int* d_ranks = nullptr;
  int* h_ranks = nullptr;  // pinned
  int* d_info = nullptr;
  slar::EigJob* d_eig = nullptr;
  slar::RankJob* d_rank = nullptr;

  // fields, moments, spectral work, LoMaC and Newton-Krylov buffers
  double* E = nullptr;       // [dx][NX] current field
  double* E1 = nullptr;
  double* E2 = nullptr;
  double* E3 = nullptr;
  double* mom = nullptr;     // [n_mom][NX]
  double* lvec = nullptr;    // leaf moment vectors
  double* spec = nullptr;    // spectral work (complex), several fields
  long long spec_len = 0;    // in doubles
  slar::Spectral* spectral = nullptr;
  double* rho = nullptr;     // [NX]
  double* Wdev = nullptr;    // device scalars (electric energy, ...)
  double* macro_ws = nullptr;
  long long macro_ws_len = 0;
  double* lomac_bs = nullptr;   // basis scalars of the closure (LS_SIZE)
  double* lomac_qv = nullptr;   // basis vectors of the closure [3][dv][Nv]
  double* lomac_C = nullptr;    // C(F*) [dv+2][NX]
  slar::MacroWS* mw = nullptr;
  double* scal = nullptr;    // device scalars for the solver
  double* scal_host = nullptr;  // pinned mirror

  // profiling of the entry evaluator (SLAR_PROFILE): event pairs around every launch
  cudaEvent_t prof_ev[2048] = {};
  int prof_n = 0;          // pairs recorded this step
  cudaEvent_t ph_ev[256] = {};  // phase boundary events (SLAR_PROFILE)
  int ph_tag[256] = {};
  int ph_n = 0;
  double prof_flop = 0.0;  // algorithmic flops of the sampled entries this step

  // learned warm start and training-sample recording
  slar_net* net = nullptr;         // attached network (not owned)
  float* rec_dst = nullptr;        // device destination of the next sample (one-shot)
  int rec_S = 0;
  unsigned long long rec_seed = 0;

  // SLAR calls and truncations that stopped at the rank cap with eps unmet (running count;
  // sl_step, slar_advect, ht_truncate and init_ht report SLAR_ERANK when it grows)
  long long rank_capped = 0;
  // block-circulant preconditioner reuse: steps since the last probe (-1: none valid), the
  // coefficient beta dt it was probed for, and the GMRES count of the solve right after it
  int pc_age = -1;
  double pc_coef = 0.0;
  int pc_krylov_ref = 0;
  bool pc_stale = false;
  int pc_off = 0;   // BDF3 steps left before the preconditioned solve is tried again

  char err[512] = {0};
};

namespace slar {

struct TruncIn {
  int d;
  int r[6];
  const double* U[4];  // nullptr = identity leaf (r[mu] == N[mu])
  const double* B12;
  const double* B34;
  const double* Broot;
  bool fast_qr;        // CholQR2 (inputs of full column rank) instead of Householder QR
};

slar_status set_error(slar_ctx* c, slar_status st, const char* msg);
slar_status cuda_fail(slar_ctx* c, cudaError_t e, const char* where);
// HSVD truncation of `in` written into slot `out_slot` (which must not be an input).
slar_status truncate_into(slar_ctx* c, const TruncIn& in, double eps, int cap, int out_slot);
TruncIn trunc_in_of_slot(const slar_ctx* c, int slot);
HTView<double> view64(const slar_ctx* c, int slot);
HTView<float> view32_slot(const slar_ctx* c, int slot);
slar_status refresh_f32_slot(slar_ctx* c, int slot);
// FP32 copies of the field E (if given) and of the LoMaC correction (if with_corr) for the
// FP32 / BF16x3 evaluators; nothing in FP64 mode
slar_status refresh_f32_fields(slar_ctx* c, const double* E, bool with_corr);
slar_status build_aca_graph(slar_ctx* c, size_t smem, bool block);
slar_status aca_step(slar_ctx* c, size_t smem, cudaGraphConditionalHandle h, int use_cond, bool prof);
slar_status aca_block_step(slar_ctx* c, size_t smem, cudaGraphConditionalHandle h, int use_cond, bool prof);

// Redirects the context's launches to its capture stream while a CUDA graph is recorded
// (capture is not possible on the legacy default stream a caller may pass).
struct CaptureScope {
  slar_ctx* c;
  cudaStream_t saved;
  explicit CaptureScope(slar_ctx* ctx);
  ~CaptureScope();
};
CorrView corr_view(const slar_ctx* c, bool with_corr);
// evaluate entries of slot (+ the state's correction if with_corr) in the context precision
slar_status eval_entries(slar_ctx* c, int slot, bool with_corr, const EvalArgs& a, int at_grid);
// one SLAR call: cross approximation of the SL update of slot `in` (+ correction), then
// truncation into slot `out`
slar_status slar_call(slar_ctx* c, int in, bool with_corr, double tau, const double* E, int out,
                      int* aca_rank, long long* entries);
// algorithmic flops of one SL entry of a slot: leaf interpolation 3 r_mu per leaf, transfer
// tensors r_t1 r_t2 r_t, root r12 r34 (multiply-adds x 2), plus 60 for foot and weights
double entry_flops(const slar_ctx* c, int slot);

// moments / fields / LoMaC / macro (see the respective .cu files)
slar_status compute_moments(slar_ctx* c, int slot, bool with_corr, double* out, int nmom);
slar_status field_from_M0(slar_ctx* c, const double* M0, double* E, double* phi, double* W_dev);
slar_status poisson_dev(slar_ctx* c, const double* rho, double* E, double* phi, double* W_dev);
slar_status lomac_apply(slar_ctx* c, const double* Utarget);
slar_status conserved_from_moments(slar_ctx* c, const double* mom, const double* E, double* U);
slar_status macro_alloc(slar_ctx* c);
void macro_free(slar_ctx* c);
slar_status step_impl(slar_ctx* c, double dt, slar_stats* st);
// variable-step BDF3 coefficients (a[3], beta) for the steps (h_n, h_{n-1}, h_{n-2})
void bdf3_variable(const double h[3], double a[3], double* beta);
// the largest ratio h_n / h_{n-1} admitted for variable-step BDF3
constexpr double kBdf3RatioMax = 1.4877;
// BDF3 steps a probed block-circulant preconditioner is kept at most
constexpr int kPcMaxAge = 8;
// BDF3 steps solved by plain JFNK after a preconditioned solve fell back to it
constexpr int kPcOffSteps = 8;
// adaptive step size: cfl / max_i(a_i / Delta_i), capped at dt_max and, after the start-up,
// at kBdf3RatioMax times the previous step (field of the current state)
slar_status cfl_dt(slar_ctx* c, double cfl, double dt_max, double* dt);

// BF16 pieces of the tensor-core evaluator in this context: 2 (BF16x3), 3 (BF16x6), or 0
// where entries are evaluated on the CUDA cores (FP64, FP32, and every d = 2 tree)
inline int tc_pieces(const slar_ctx* c) {
  if (c->d != 4) return 0;
  return c->cfg.precision == SLAR_FP32_BF16X3 ? 2 : c->cfg.precision == SLAR_FP32_BF16X6 ? 3 : 0;
}

}  // namespace slar

#define CK(call)                                               \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return slar::cuda_fail(c, e_, #call); \
  } while (0)
#define CKS(call)                      \
  do {                                 \
    slar_status s_ = (call);           \
    if (s_ != SLAR_OK) return s_;      \
  } while (0)
