// Cross approximation of the SL-updated tensor (the HTACA step of SLAR, Sec. 3.1): the
// matricisation A = F_(x | v) is approximated by U V^T from sampled row and column fibres,
// with partial pivoting; then the exact HT embedding and the HSVD truncation.
//
// Reading of the paper (which defers HTACA to earlier work): partially pivoted ACA on the
// root split, start row 0, stop when ||u_k|| ||v_k|| <= eps ||A_k||_F (running estimate)
// or k = cap; arg-max ties within a relative 1e-10 go to the lowest index.
//
// Every step runs on the device with no host round trip: the entry evaluator samples the
// residual row (fused residual epilogue), one CTA picks the column pivot and scales v_k,
// the evaluator samples the residual column into u_k, a grid kernel forms the dot products
// of the norm estimate, and one CTA updates the estimate, tests the stop rule and picks the
// next row pivot.  A device flag makes the remaining launches of a stopped approximation
// exit immediately; the host reads the final rank once.
#include "context.cuh"

namespace slar {
namespace {

constexpr int PIV_THREADS = 1024;
constexpr int DOT_SEG = 256;
constexpr double TIE_RTOL = 1e-10;

__device__ void block_argmax_tie(const double* a, int n, const unsigned char* used, int* out_idx,
                                 double* out_max) {
  // two passes: global max of |a| over unused, then the lowest index within the tie band
  __shared__ double wmax[PIV_THREADS / 32];
  __shared__ int widx[PIV_THREADS / 32];
  __shared__ double top_s;
  const int tid = threadIdx.x;
  double m = -1.0;
  for (int i = tid; i < n; i += PIV_THREADS)
    if (!used[i]) m = fmax(m, fabs(a[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) wmax[tid >> 5] = m;
  __syncthreads();
  if (tid == 0) {
    double t = -1.0;
    for (int w = 0; w < PIV_THREADS / 32; ++w) t = fmax(t, wmax[w]);
    top_s = t;
  }
  __syncthreads();
  const double top = top_s;
  const double thr = top * (1.0 - TIE_RTOL);
  int best = 0x7fffffff;
  if (top >= 0.0)
    for (int i = tid; i < n; i += PIV_THREADS)
      if (!used[i] && fabs(a[i]) >= thr && i < best) best = i;
  for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_down_sync(0xffffffffu, best, o));
  if ((tid & 31) == 0) widx[tid >> 5] = best;
  __syncthreads();
  if (tid == 0) {
    int b = 0x7fffffff;
    for (int w = 0; w < PIV_THREADS / 32; ++w) b = min(b, widx[w]);
    *out_idx = (top >= 0.0 && b != 0x7fffffff) ? b : -1;
    *out_max = top;
  }
  __syncthreads();
}

__global__ void k_aca_init(AcaState* st, int* pivI, unsigned char* usedr, int replay) {
  if (threadIdx.x != 0) return;
  st->k = 0;
  st->done = 0;
  st->stop_row = 0;
  st->normA2 = 0.0;
  if (!replay) pivI[0] = 0;
  if (pivI[0] < 0) { st->done = 1; return; }
  usedr[pivI[0]] = 1;
}

// column pivot from the residual row r, v_k = r / r[j_k]
__global__ void __launch_bounds__(PIV_THREADS)
k_aca_row_pivot(const double* __restrict__ r, int M2, unsigned char* usedc, int* pivJ, int kk,
                AcaState* st, double* __restrict__ vout, int replay) {
  __shared__ int j_s;
  __shared__ double top_s;
  if (st->done) return;
  if (replay) {
    if (threadIdx.x == 0) { j_s = pivJ[kk]; top_s = 1.0; }
    __syncthreads();
  } else {
    block_argmax_tie(r, M2, usedc, &j_s, &top_s);
  }
  const int j = j_s;
  if (j < 0 || top_s == 0.0 || r[j] == 0.0) {
    if (threadIdx.x == 0) { st->done = 1; st->stop_row = replay ? 0 : 1; }
    return;
  }
  const double piv = r[j];
  for (int i = threadIdx.x; i < M2; i += PIV_THREADS) vout[i] = r[i] / piv;
  if (threadIdx.x == 0) {
    pivJ[kk] = j;
    usedc[j] = 1;
    st->piv = piv;
  }
}

// partial dot products of u_k with U_l (l < kk) and itself, v_k with V_l and itself
__global__ void __launch_bounds__(256)
k_aca_dots(const double* __restrict__ Ua, int M1, const double* __restrict__ Va, int M2, int kk,
           int nbu, const AcaState* st, double* __restrict__ part, int ldp) {
  if (st->done) return;
  const int blk = blockIdx.x;
  const bool isu = blk < nbu;
  const double* X = isu ? Ua : Va;
  const int M = isu ? M1 : M2;
  const int s0 = (isu ? blk : blk - nbu) * DOT_SEG;
  const double* xk = X + (long long)kk * M;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int l = warp; l <= kk; l += 8) {
    const double* xl = X + (long long)l * M;
    double acc = 0.0;
    for (int i = s0 + lane; i < s0 + DOT_SEG && i < M; i += 32) acc += xl[i] * xk[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) part[(long long)blk * ldp + l] = acc;
  }
}

// norm estimate, stop test, next row pivot
__global__ void __launch_bounds__(PIV_THREADS)
k_aca_finalize(const double* __restrict__ Ua, int M1, int kk, int kmax, int nbu, int nbv,
               const double* __restrict__ part, int ldp, AcaState* st, int* pivI,
               unsigned char* usedr, double eps, int replay) {
  __shared__ double du[SLAR_MAX_RANK + 1], dv[SLAR_MAX_RANK + 1];
  __shared__ int i_s;
  __shared__ double top_s;
  __shared__ int stop_s;
  if (st->done) return;
  const int tid = threadIdx.x;
  if (tid <= kk) {
    double a = 0.0, b = 0.0;
    for (int blk = 0; blk < nbu; ++blk) a += part[(long long)blk * ldp + tid];
    for (int blk = nbu; blk < nbu + nbv; ++blk) b += part[(long long)blk * ldp + tid];
    du[tid] = a;
    dv[tid] = b;
  }
  __syncthreads();
  if (tid == 0) {
    double cross = 0.0;
    for (int l = 0; l < kk; ++l) cross += du[l] * dv[l];
    const double nu2 = du[kk], nv2 = dv[kk];
    const double n2 = st->normA2 + 2.0 * cross + nu2 * nv2;
    st->normA2 = n2;
    st->k = kk + 1;
    int stop = 0;
    if (kk + 1 >= kmax) stop = 1;
    else if (!replay && sqrt(nu2) * sqrt(nv2) <= eps * sqrt(fmax(n2, 0.0))) stop = 1;
    else if (replay && pivI[kk + 1] < 0) stop = 1;
    if (stop) st->done = 1;
    stop_s = stop;
  }
  __syncthreads();
  if (stop_s) return;
  if (replay) {
    if (tid == 0) usedr[pivI[kk + 1]] = 1;
    return;
  }
  block_argmax_tie(Ua + (long long)kk * M1, M1, usedr, &i_s, &top_s);
  if (tid == 0) {
    if (i_s < 0) {
      st->done = 1;
    } else {
      pivI[kk + 1] = i_s;
      usedr[i_s] = 1;
    }
  }
}

}  // namespace

slar_status slar_call(slar_ctx* c, int in, bool with_corr, double tau, const double* E, int out,
                      int* aca_rank, long long* entries) {
  cudaStream_t s = c->s;
  const int M1 = c->M1, M2 = c->M2;
  const int kmax = c->kmax;
  if (in == out) return set_error(c, SLAR_EINVAL, "SLAR output slot equals input slot");
  const bool replay = c->replay_pos < c->replay_calls;
  phase(c, PH_ACA);
  CK(cudaMemsetAsync(c->usedr, 0, M1, s));
  CK(cudaMemsetAsync(c->usedc, 0, M2, s));
  if (replay) {
    std::vector<int> I(kmax, -1), J(kmax, -1);
    const int* src = c->replay.data() + (size_t)c->replay_pos * c->replay_kmax * 2;
    for (int k = 0; k < kmax && k < c->replay_kmax; ++k) {
      I[k] = src[2 * k];
      J[k] = src[2 * k + 1];
      if (I[k] < 0 || J[k] < 0) { I[k] = J[k] = -1; break; }
      if (I[k] >= M1 || J[k] >= M2)
        return set_error(c, SLAR_EINVAL, "replayed pivot outside the matricisation");
    }
    CK(cudaMemcpy(c->pivI, I.data(), sizeof(int) * kmax, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->pivJ, J.data(), sizeof(int) * kmax, cudaMemcpyHostToDevice));
    c->replay_pos++;
  }
  slar::count_launch(), k_aca_init<<<1, 32, 0, s>>>(c->ast, c->pivI, c->usedr, replay ? 1 : 0);
  CK(cudaGetLastError());
  const int nbu = (M1 + DOT_SEG - 1) / DOT_SEG, nbv = (M2 + DOT_SEG - 1) / DOT_SEG;
  const int ldp = SLAR_MAX_RANK + 1;
  for (int kk = 0; kk < kmax; ++kk) {
    EvalArgs ar{};
    ar.mode = EVAL_ROW;
    ar.n = M2;
    ar.pivot = c->pivI + kk;
    ar.done = &c->ast->done;
    ar.kterms = kk;
    ar.X = c->Ua;
    ar.ldX = M1;
    ar.Y = c->Va;
    ar.ldY = M2;
    ar.out = c->rowbuf;
    ar.tau = tau;
    ar.E = E;
    ar.foot_euler = (c->cfg.flags & SLAR_FOOT_EULER) ? 1 : 0;
    CKS(eval_entries(c, in, with_corr, ar, 0));
    slar::count_launch(), k_aca_row_pivot<<<1, PIV_THREADS, 0, s>>>(c->rowbuf, M2, c->usedc, c->pivJ, kk, c->ast,
                                              c->Va + (long long)kk * M2, replay ? 1 : 0);
    CK(cudaGetLastError());
    EvalArgs ac = ar;
    ac.mode = EVAL_COL;
    ac.n = M1;
    ac.pivot = c->pivJ + kk;
    ac.X = c->Va;
    ac.ldX = M2;
    ac.Y = c->Ua;
    ac.ldY = M1;
    ac.out = c->Ua + (long long)kk * M1;
    CKS(eval_entries(c, in, with_corr, ac, 0));
    slar::count_launch(), k_aca_dots<<<nbu + nbv, 256, 0, s>>>(c->Ua, M1, c->Va, M2, kk, nbu, c->ast, c->aca_part, ldp);
    CK(cudaGetLastError());
    slar::count_launch(), k_aca_finalize<<<1, PIV_THREADS, 0, s>>>(c->Ua, M1, kk, kmax, nbu, nbv, c->aca_part, ldp,
                                             c->ast, c->pivI, c->usedr, c->cfg.eps, replay ? 1 : 0);
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(c->ast_host, c->ast, sizeof(AcaState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const int k = c->ast_host->k;
  if (aca_rank) *aca_rank = k;
  const long long nent = (long long)k * (M1 + M2) + (c->ast_host->stop_row ? M2 : 0);
  if (entries) *entries = nent;
  c->prof_flop += (double)nent * entry_flops(c, in);
  if (k == 0) return set_error(c, SLAR_ENAN, "cross approximation found no pivot (zero tensor)");
  // exact HT embedding of U V^T, then HSVD truncation
  phase(c, PH_TRUNC);
  TruncIn tin;
  tin.d = c->d;
  tin.fast_qr = true;
  if (c->d == 4) {
    for (int m = 0; m < 4; ++m) {
      tin.U[m] = nullptr;
      tin.r[m] = c->g.N[m];
    }
    tin.r[4] = tin.r[5] = k;
    tin.B12 = c->Ua;
    tin.B34 = c->Va;
  } else {
    CK(transpose(c->Ua, k, M1, c->Lt[0], s));
    CK(transpose(c->Va, k, M2, c->Lt[1], s));
    tin.U[0] = c->Lt[0];
    tin.U[1] = c->Lt[1];
    tin.U[2] = tin.U[3] = nullptr;
    tin.r[0] = tin.r[1] = k;
    tin.r[2] = tin.r[3] = tin.r[4] = tin.r[5] = 0;
    tin.B12 = tin.B34 = nullptr;
  }
  CK(fill_identity(c->Ik, k, k, s));
  tin.Broot = c->Ik;
  return truncate_into(c, tin, c->cfg.eps, c->cfg.rank_cap, out);
}

}  // namespace slar
