// HT state management on the device: HSVD truncation (Supp. B.1), the FP32 shadow,
// entry evaluation wrappers, initial data from separable terms, import / export.
#include <cstdio>
#include <cstring>

#include "context.cuh"

namespace slar {

slar_status set_error(slar_ctx* c, slar_status st, const char* msg) {
  if (c) snprintf(c->err, sizeof(c->err), "%s", msg);
  return st;
}

slar_status cuda_fail(slar_ctx* c, cudaError_t e, const char* where) {
  if (c) snprintf(c->err, sizeof(c->err), "CUDA error %s (%s) at %s", cudaGetErrorName(e),
                  cudaGetErrorString(e), where);
  return e == cudaErrorMemoryAllocation ? SLAR_ENOMEM : SLAR_ECUDA;
}

HTView<double> view64(const slar_ctx* c, int slot) {
  HTView<double> v;
  const HTBuf& h = c->ht[slot];
  for (int m = 0; m < 4; ++m) {
    v.U[m] = h.U[m];
    v.r[m] = h.r[m];
  }
  v.B12 = h.B12;
  v.B34 = h.B34;
  v.Broot = h.Broot;
  v.r12 = h.r[4];
  v.r34 = h.r[5];
  return v;
}

HTView<float> view32_slot(const slar_ctx* c, int slot) {
  HTView<float> v;
  const HTBuf& h = c->ht[slot];
  for (int m = 0; m < 4; ++m) {
    v.U[m] = c->U32[m];
    v.r[m] = h.r[m];
  }
  v.B12 = c->B12_32;
  v.B34 = c->B34_32;
  v.Broot = c->Broot32;
  v.r12 = h.r[4];
  v.r34 = h.r[5];
  return v;
}

CorrView corr_view(const slar_ctx* c, bool with_corr) {
  CorrView v;
  v.dC = c->dC;
  v.qv = c->qv;
  v.dC32 = c->dC32;
  v.qv32 = c->qv32;
  v.has = (with_corr && c->has_corr) ? 1 : 0;
  return v;
}

// FP32 copy of a slot's factors for the FP32 entry evaluator.
slar_status refresh_f32_slot(slar_ctx* c, int slot) {
  if (c->f32_slot == slot) return SLAR_OK;
  const HTBuf& h = c->ht[slot];
  F32Batch bt;
  for (int m = 0; m < c->d; ++m) bt.add(h.U[m], c->U32[m], (long long)c->g.N[m] * h.r[m]);
  if (c->d == 4) {
    bt.add(h.B12, c->B12_32, (long long)h.r[4] * h.r[0] * h.r[1]);
    bt.add(h.B34, c->B34_32, (long long)h.r[5] * h.r[2] * h.r[3]);
    bt.add(h.Broot, c->Broot32, (long long)h.r[4] * h.r[5]);
    CK(to_float_batch(bt, c->s));
    if (tc_pieces(c) > 0) {
      CK(split_transfer_bf16(c->B12_32, h.r[4], h.r[0], h.r[1], c->tc_b12, tc_pieces(c), c->s));
      CK(split_transfer_bf16(c->B34_32, h.r[5], h.r[2], h.r[3], c->tc_b34, tc_pieces(c), c->s));
      CK(split_root_bf16(c->Broot32, h.r[4], h.r[5], c->tc_broot, tc_pieces(c), c->s));
    }
  } else {
    bt.add(h.Broot, c->Broot32, (long long)h.r[0] * h.r[1]);
    CK(to_float_batch(bt, c->s));
  }
  c->f32_slot = slot;
  return SLAR_OK;
}

slar_status refresh_f32_fields(slar_ctx* c, const double* E, bool with_corr) {
  if (c->cfg.precision == SLAR_FP64) return SLAR_OK;
  F32Batch bt;
  if (E) bt.add(E, c->E32, (long long)c->dx * c->NX);
  if (with_corr && c->has_corr) {
    bt.add(c->dC, c->dC32, (long long)(c->dv + 2) * c->NX);
    bt.add(c->qv, c->qv32, (long long)3 * c->dv * c->g.N[c->dx]);
  }
  CK(to_float_batch(bt, c->s));
  return SLAR_OK;
}

CaptureScope::CaptureScope(slar_ctx* ctx) : c(ctx), saved(ctx->s) {
  c->s = c->cap_s;
  c->spectral->s = c->cap_s;
}

CaptureScope::~CaptureScope() {
  c->s = saved;
  c->spectral->s = saved;
}

void phase(slar_ctx* c, int tag) {
  if (!(c->cfg.flags & SLAR_PROFILE) || c->ph_n >= kPhaseEvents) return;
  if (cudaEventRecord(c->ph_ev[c->ph_n], c->s) == cudaSuccess) c->ph_tag[c->ph_n++] = tag;
}

double entry_flops(const slar_ctx* c, int slot) {
  const int* r = c->ht[slot].r;
  double f = 0.0;
  for (int m = 0; m < c->d; ++m) f += 3.0 * r[m];
  if (c->d == 4) f += (double)r[0] * r[1] * r[4] + (double)r[2] * r[3] * r[5] + (double)r[4] * r[5];
  else f += (double)r[0] * r[1];
  return 2.0 * f + 60.0;
}

slar_status eval_entries(slar_ctx* c, int slot, bool with_corr, const EvalArgs& a, int at_grid) {
  if (!c->ht[slot].valid) return set_error(c, SLAR_EINVAL, "no HT state");
  const bool prof = (c->cfg.flags & SLAR_PROFILE_EVAL) && c->prof_n * 2 + 1 < kProfEvents;
  if (prof) CK(cudaEventRecord(c->prof_ev[2 * c->prof_n], c->s));
  cudaError_t e;
  EvalArgs b = a;
  b.E32 = c->E32;   // refreshed by the caller (refresh_f32_fields)
  if (tc_pieces(c) > 0 && !at_grid) {
    CKS(refresh_f32_slot(c, slot));
    e = launch_sl_eval_tc(c->g, view32_slot(c, slot), corr_view(c, with_corr), b, c->tc_b12, c->tc_b34,
                          c->tc_broot, &c->ast->tc_err, tc_pieces(c), c->tc_sc, c->s);
  } else if (c->cfg.precision != SLAR_FP64) {
    CKS(refresh_f32_slot(c, slot));
    c->eval_tile = sl_eval_fit_tile<float>(c->g, c->ht[slot].r, c->eval_tile);
    e = launch_sl_eval<float>(c->g, view32_slot(c, slot), corr_view(c, with_corr), b, at_grid, c->s, c->eval_tile);
  } else {
    c->eval_tile = sl_eval_fit_tile<double>(c->g, c->ht[slot].r, c->eval_tile);
    e = launch_sl_eval<double>(c->g, view64(c, slot), corr_view(c, with_corr), a, at_grid, c->s, c->eval_tile);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "sl_eval kernel");
  if (prof) {
    CK(cudaEventRecord(c->prof_ev[2 * c->prof_n + 1], c->s));
    c->prof_n++;
  }
  return SLAR_OK;
}

TruncIn trunc_in_of_slot(const slar_ctx* c, int slot) {
  const HTBuf& h = c->ht[slot];
  TruncIn in;
  in.d = c->d;
  for (int i = 0; i < 6; ++i) in.r[i] = h.r[i];
  for (int m = 0; m < 4; ++m) in.U[m] = h.U[m];
  in.B12 = h.B12;
  in.B34 = h.B34;
  in.Broot = h.Broot;
  in.fast_qr = false;
  return in;
}

namespace {

__global__ void k_trace(const double* G, int n, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += G[i * n + i];
    out[0] = s;
  }
}

// QR of a column-major m x n matrix A (not modified): Q column-major m x n, R n x n.
slar_status qr_colmajor(slar_ctx* c, const double* A, int m, int n, double* Q, double* R,
                        bool fast) {
  cudaStream_t s = c->s;
  if (!fast) {
    CK(cudaMemcpyAsync(c->T3, A, sizeof(double) * (size_t)m * n, cudaMemcpyDeviceToDevice, s));
    CK(householder_qr(c->T3, m, n, Q, R, c->tau, s));
    return SLAR_OK;
  }
  // CholQR2 with column equilibration: A = Q1 R1, Q1 = Q R2, R = R2 R1
  double* G = c->sm1;
  double* R1 = c->sm2;
  double* R1i = c->sm3;
  double* R2 = c->sm4;
  CK(gram_tall(A, m, m, n, G, c->gram_work, c->gram_work_blocks, s));
  CK(chol_inv(G, n, R1, R1i, c->d_info, s));
  // Q1^T (n x m row-major) = R1inv^T A^T
  CK(dgemm(1, 0, n, m, n, 1.0, R1i, n, 0, A, m, 0, 0.0, c->T3, m, 0, 1, s));
  CK(gram_tall(c->T3, m, m, n, G, c->gram_work, c->gram_work_blocks, s));
  CK(chol_inv(G, n, R2, R1i, c->d_info + 1, s));
  CK(dgemm(1, 0, n, m, n, 1.0, R1i, n, 0, c->T3, m, 0, 0.0, Q, m, 0, 1, s));
  CK(dgemm(0, 0, n, n, n, 1.0, R2, n, 0, R1, n, 0, 0.0, R, n, 0, 1, s));
  return SLAR_OK;
}

}  // namespace

// HSVD truncation of the input HT, written into slot out_slot.
slar_status truncate_into(slar_ctx* c, const TruncIn& in, double eps, int cap, int out_slot) {
  cudaStream_t s = c->s;
  const int d = in.d;
  const int* N = c->g.N;
  HTBuf& out = c->ht[out_slot];
  if (c->f32_slot == out_slot) c->f32_slot = -1;
  int rq[4];          // leaf ranks after orthogonalisation
  bool ident[4];
  CK(cudaMemsetAsync(c->d_info, 0, sizeof(int) * 2, s));
  // 1. leaves: Q_mu (row-major N x r) and R_mu (r x r)
  for (int m = 0; m < d; ++m) {
    ident[m] = (in.U[m] == nullptr);
    rq[m] = in.r[m];
    if (ident[m]) continue;
    if (in.r[m] > N[m]) return set_error(c, SLAR_EINVAL, "leaf rank exceeds grid size");
    // column-major view of the leaf = transpose of the row-major N x r array
    CK(transpose(in.U[m], N[m], in.r[m], c->T1, s));
    CKS(qr_colmajor(c, c->T1, N[m], in.r[m], c->T2, c->Rleaf[m], in.fast_qr));
    CK(transpose(c->T2, in.r[m], N[m], c->Qleaf[m], s));
  }
  double* Bq[2] = {c->Q12, c->Q34};
  double* Broot1 = c->sm1;
  if (d == 2) {
    // Broot' = R0 Broot R1^T
    const int r0 = in.r[0], r1 = in.r[1];
    CK(dgemm(0, 0, r0, r1, r0, 1.0, c->Rleaf[0], r0, 0, in.Broot, r1, 0, 0.0, c->sm2, r1, 0, 1, s));
    CK(dgemm(0, 1, r0, r1, r1, 1.0, c->sm2, r1, 0, c->Rleaf[1], r1, 0, 0.0, Broot1, r1, 0, 1, s));
    CK(dgemm(0, 1, r0, r0, r1, 1.0, Broot1, r1, 0, Broot1, r1, 0, 0.0, c->G[0], r0, 0, 1, s));
    CK(dgemm(1, 0, r1, r1, r0, 1.0, Broot1, r1, 0, Broot1, r1, 0, 0.0, c->G[1], r1, 0, 1, s));
  } else {
    const double* Bin[2] = {in.B12, in.B34};
    for (int t = 0; t < 2; ++t) {
      const int a = 2 * t, b = 2 * t + 1;
      const int ra = rq[a], rb = rq[b], rp = in.r[4 + t];
      const long long K = (long long)ra * rb;
      const double* B = Bin[t];
      if (!ident[a] || !ident[b]) {
        // B'_p = R_a B_p R_b^T (identity leaves contribute R = I)
        const double* Ra = ident[a] ? nullptr : c->Rleaf[a];
        const double* Rb = ident[b] ? nullptr : c->Rleaf[b];
        const double* src = B;
        if (Ra) {
          CK(dgemm(0, 0, ra, rb, ra, 1.0, Ra, ra, 0, src, rb, K, 0.0, c->T1, rb, K, rp, s));
          src = c->T1;
        }
        if (Rb) {
          CK(dgemm(0, 1, ra, rb, rb, 1.0, src, rb, K, Rb, rb, 0, 0.0, c->T2, rb, K, rp, s));
          src = c->T2;
        }
        if (src != c->T2) CK(cudaMemcpyAsync(c->T2, src, sizeof(double) * K * rp,
                                             cudaMemcpyDeviceToDevice, s));
        B = c->T2;
      }
      // QR of B as a column-major K x rp matrix
      CKS(qr_colmajor(c, B, (int)K, rp, Bq[t], c->Rn[t], in.fast_qr));
    }
    // Broot' = R12 Broot R34^T
    const int r12 = in.r[4], r34 = in.r[5];
    CK(dgemm(0, 0, r12, r34, r12, 1.0, c->Rn[0], r12, 0, in.Broot, r34, 0, 0.0, c->sm2, r34, 0, 1, s));
    CK(dgemm(0, 1, r12, r34, r34, 1.0, c->sm2, r34, 0, c->Rn[1], r34, 0, 0.0, Broot1, r34, 0, 1, s));
    // node Gram matrices, root down
    CK(dgemm(0, 1, r12, r12, r34, 1.0, Broot1, r34, 0, Broot1, r34, 0, 0.0, c->G[4], r12, 0, 1, s));
    CK(dgemm(1, 0, r34, r34, r12, 1.0, Broot1, r34, 0, Broot1, r34, 0, 0.0, c->G[5], r34, 0, 1, s));
    for (int t = 0; t < 2; ++t) {
      const int a = 2 * t, b = 2 * t + 1;
      const int ra = rq[a], rb = rq[b], rp = in.r[4 + t];
      const long long K = (long long)ra * rb;
      // T[p'][a][b] = sum_p G[p][p'] B[p][a][b]
      CK(dgemm(0, 0, rp, (int)K, rp, 1.0, c->G[4 + t], rp, 0, Bq[t], (int)K, 0, 0.0, c->T1,
               (int)K, 0, 1, s));
      const long long wl = (long long)c->gram_work_blocks * SLAR_MAX_RANK * SLAR_MAX_RANK;
      CK(contract_last(c->T1, Bq[t], rp, ra, ra, rb, c->G[a], c->gram_work, wl, s));
      CK(contract_mid(c->T1, Bq[t], rp, ra, rb, rb, c->G[b], c->gram_work, wl, s));
    }
  }
  // 2. eigendecompositions.  Leaf Gram matrices of the same order as at the previous
  // truncation are first rotated into the previous eigenbasis, A' = S^T G S, which is
  // nearly diagonal because the distribution changes little between SLAR calls; Jacobi then
  // needs far fewer sweeps and the eigenvectors are S V'.
  EigJob jobs[6];
  int nj = 0;
  int node_n[6];
  for (int m = 0; m < d; ++m) node_n[m] = rq[m];
  if (d == 4) { node_n[4] = in.r[4]; node_n[5] = in.r[5]; }
  const int nnodes = d == 4 ? 6 : 2;
  bool warm[6] = {false, false, false, false, false, false};
  // Gram matrices above order 24 are compressed before the eigen-solve (k_jacobi: pivoted
  // Cholesky down to the numerical range, Jacobi of that order, hand-over to the
  // tridiagonal solver above rank 40).  FP32 / BF16x3 data: the dropped trace is 1/10 of the
  // rank threshold.  FP64 data: 1e-16 of the trace, the rounding level of a Gram matrix --
  // the eigenvalues dropped there are the ones a dense solver (LAPACK's, the oracle's) also
  // resolves only to about u ||G||, and the kept eigenvectors move by ~u ||G|| / gap: the
  // truncated tensor by ~u / sqrt(threshold) of ||F||, at most 1e-10 (a tenth of the FP64
  // parity bar) for the rank thresholds eps^2 / (2d - 3) >= 1e-12 it is used at.
  const double thr_rel = eps * eps / (2.0 * d - 3.0);
  const bool fp64 = c->cfg.precision == SLAR_FP64;
  auto compress_rel_of = [&](int n) {
    if (n <= 24) return 0.0;
    if (fp64) return thr_rel >= 1e-12 ? 1e-16 : 0.0;
    return std::max(1e-16, 0.1 * thr_rel);
  };
  for (int m = 0; m < d; ++m) {
    const int nm = node_n[m];
    // (no warm start with the compressed eigen-solve: its basis holds only the numerical
    // range, and rotating the next Gram matrix into it would lose every new direction)
    if (nm < 16 || c->Sn[m] != nm || compress_rel_of(nm) > 0.0) continue;
    double* T = c->Sw + (size_t)m * SLAR_MAX_N * SLAR_MAX_N;
    CK(dgemm(0, 0, nm, nm, nm, 1.0, c->G[m], nm, 0, c->S[m], nm, 0, 0.0, T, nm, 0, 1, s));
    CK(dgemm(1, 0, nm, nm, nm, 1.0, c->S[m], nm, 0, T, nm, 0, 0.0, c->G[m], nm, 0, 1, s));
    // keep the previous basis in T for the back-rotation
    CK(cudaMemcpyAsync(T, c->S[m], sizeof(double) * nm * nm, cudaMemcpyDeviceToDevice, s));
    warm[m] = true;
  }
  for (int t = 0; t < nnodes; ++t) {
    jobs[nj].A = c->G[t];
    jobs[nj].W = c->W[t];
    jobs[nj].V = c->S[t];
    jobs[nj].work = c->ework[t];
    jobs[nj].n = node_n[t];
    // entries below the data noise of the Gram matrix are not rotated -- FP64 rounding
    // (1e-17), FP32 entries (u^2 ~ 4e-15: 1e-13), BF16x3 entries (about 2^-16 per product:
    // 1e-9) -- but never at or above the rank threshold eps^2/(2d-3) of the truncation: the
    // floor stays at 1/100 of it so that the eigenvalues that decide the ranks are resolved;
    // and never below the FP64 rounding level
    const double noise = c->cfg.precision == SLAR_FP64 ? 1e-17 : (c->cfg.precision == SLAR_FP32 ? 1e-13 : 1e-9);
    jobs[nj].floor_rel = std::max(1e-17, std::min(noise, 1e-2 * eps * eps / (2.0 * d - 3.0)));
    // eigen-solve only the numerical range of the Gram matrix: a pivoted Cholesky G ~ L L^T
    // stopped when the trace left out is below compress_rel trace G, then Jacobi on L^T L
    jobs[nj].compress_rel = compress_rel_of(node_n[t]);
    // the truncation reads at most cap leading eigenvectors of each node; a compressed
    // numerical rank above 40 goes to the tridiagonal path
    jobs[nj].nvec = std::min(node_n[t], cap);
    jobs[nj].tri = (jobs[nj].compress_rel > 0.0 && node_n[t] > 40) ? 1 : 0;
    ++nj;
  }
  CK(eig_batched(jobs, nj, c->d_eig, s));
  for (int m = 0; m < d; ++m) {
    if (warm[m]) {
      const int nm = node_n[m];
      double* T = c->Sw + (size_t)m * SLAR_MAX_N * SLAR_MAX_N;
      // S <- S_prev V'  (through the Jacobi scratch, free again after the solve)
      CK(dgemm(0, 0, nm, nm, nm, 1.0, T, nm, 0, c->S[m], nm, 0, 0.0, c->ework[m], nm, 0, 1, s));
      CK(cudaMemcpyAsync(c->S[m], c->ework[m], sizeof(double) * nm * nm, cudaMemcpyDeviceToDevice, s));
    }
  }
  for (int t = 0; t < nnodes; ++t) c->Sn[t] = compress_rel_of(node_n[t]) > 0.0 ? 0 : node_n[t];
  // 3. ranks
  slar::count_launch(), k_trace<<<1, 32, 0, s>>>(c->G[d == 4 ? 4 : 0], node_n[d == 4 ? 4 : 0], c->norm2);
  CK(cudaGetLastError());
  RankJob rj[5];
  int nr = 0;
  for (int m = 0; m < d; ++m) rj[nr++] = RankJob{c->W[m], node_n[m], cap, c->d_ranks + m, c->d_ranks + 6};
  if (d == 4) rj[nr++] = RankJob{c->W[4], node_n[4], cap, c->d_ranks + 4, c->d_ranks + 6};
  CK(cudaMemsetAsync(c->d_ranks + 6, 0, sizeof(int), s));
  CK(choose_ranks(rj, nr, c->d_rank, c->norm2, eps * eps / (2.0 * d - 3.0), s));
  CK(cudaMemcpyAsync(c->h_ranks, c->d_ranks, sizeof(int) * 7, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(c->h_ranks + 8, c->d_info, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (in.fast_qr && (c->h_ranks[8] != 0 || c->h_ranks[9] != 0))
    return set_error(c, SLAR_ENAN, "Cholesky-QR breakdown in truncation (rank-deficient factor)");
  if (c->h_ranks[6]) c->rank_capped++;
  int k[6];
  for (int m = 0; m < d; ++m) k[m] = c->h_ranks[m];
  if (d == 2) {
    k[0] = k[0] < node_n[1] ? k[0] : node_n[1];
    k[1] = k[0];
  } else {
    k[4] = c->h_ranks[4];
    if (k[4] > node_n[5]) k[4] = node_n[5];
    k[5] = k[4];
  }
  // 4. projection into the output buffers
  for (int m = 0; m < d; ++m) {
    if (ident[m]) {
      CK(copy_cols(c->S[m], node_n[m], N[m], k[m], out.U[m], k[m], s));
    } else {
      CK(dgemm(0, 0, N[m], k[m], rq[m], 1.0, c->Qleaf[m], rq[m], 0, c->S[m], node_n[m], 0, 0.0,
               out.U[m], k[m], 0, 1, s));
    }
  }
  if (d == 2) {
    const int r0 = rq[0], r1 = rq[1];
    CK(dgemm(1, 0, k[0], r1, r0, 1.0, c->S[0], r0, 0, Broot1, r1, 0, 0.0, c->sm2, r1, 0, 1, s));
    CK(dgemm(0, 0, k[0], k[1], r1, 1.0, c->sm2, r1, 0, c->S[1], r1, 0, 0.0, out.Broot, k[1], 0, 1, s));
  } else {
    double* Bout[2] = {out.B12, out.B34};
    for (int t = 0; t < 2; ++t) {
      const int a = 2 * t, b = 2 * t + 1;
      const int ra = rq[a], rb = rq[b], rp = in.r[4 + t];
      const long long K = (long long)ra * rb;
      const int kp = k[4 + t];
      // C[z] = sum_p S[p][z] B[p]
      CK(dgemm(1, 0, kp, (int)K, rp, 1.0, c->S[4 + t], rp, 0, Bq[t], (int)K, 0, 0.0, c->T1,
               (int)K, 0, 1, s));
      // E_z = S_a^T C_z   (k_a x rb)
      CK(dgemm(1, 0, k[a], rb, ra, 1.0, c->S[a], ra, 0, c->T1, rb, K, 0.0, c->T2, rb,
               (long long)k[a] * rb, kp, s));
      // D_z = E_z S_b[:, :k_b]
      CK(dgemm(0, 0, k[a], k[b], rb, 1.0, c->T2, rb, (long long)k[a] * rb, c->S[b], rb, 0, 0.0,
               Bout[t], k[b], (long long)k[a] * k[b], kp, s));
    }
    const int r12 = in.r[4], r34 = in.r[5];
    CK(dgemm(1, 0, k[4], r34, r12, 1.0, c->S[4], r12, 0, Broot1, r34, 0, 0.0, c->sm2, r34, 0, 1, s));
    CK(dgemm(0, 0, k[4], k[5], r34, 1.0, c->sm2, r34, 0, c->S[5], r34, 0, 0.0, out.Broot, k[5], 0, 1, s));
  }
  for (int m = 0; m < d; ++m) out.r[m] = k[m];
  if (d == 4) { out.r[4] = k[4]; out.r[5] = k[5]; } else { out.r[4] = out.r[5] = 0; }
  out.valid = true;
  return SLAR_OK;
}

}  // namespace slar
