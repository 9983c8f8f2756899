// Internal declarations shared by the CUDA translation units of libslar.so.
// Device layouts (all row-major):
//   leaf U_mu            : N_mu x r_mu        (row = grid index, ranks contiguous)
//   B12 / B34            : [p][a][b]          (r12 x r0 x r1 / r34 x r2 x r3)
//   Broot                : r0 x r1 (d = 2) or r12 x r34 (d = 4)
//   cross factors Ua, Va : column-major M1 x kmax / M2 x kmax (column k contiguous)
// With this choice a d = 4 cross factor Ua *is* a transfer tensor [p][(a,b)] for identity
// leaves, so the exact HT embedding of the cross approximation costs no copy.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "../../include/slar.h"

#define SLAR_MAX_RANK 64
#define SLAR_MAX_N 128

namespace slar {

// Number of kernels this library has launched (all contexts); every launch site bumps it.
long long launch_count();
int count_launch();
void add_launches(long long n);  // kernels executed by a replayed CUDA graph

struct GridDesc {
  int d, dx, dv;
  int N[4];
  double lo[4], h[4];
  double ih[4];          // 1 / h (FP64)
  float lof[4], hf[4];   // the same in FP32 (the FP32 / BF16 paths' arithmetic)
  float ihf[4];          // 1 / h rounded to FP32
  int NX;  // prod of spatial N
  int NV;  // prod of velocity N
  int S;   // interpolation stencil points per dimension: 3 (quadratic) or 5 (quartic, FP64)
};

template <typename T>
struct HTView {
  const T* U[4];
  int r[4];
  const T* B12;
  const T* B34;
  const T* Broot;
  int r12, r34;
};

struct CorrView {
  const double* dC;  // [dv+2][NX]
  const double* qv;  // [3][dv][Nv]  omega, q1, q2 per velocity dim
  const float* dC32; // FP32 copies for the FP32 / BF16x3 paths
  const float* qv32;
  int has;
};

// What the entry evaluator computes for each entry e of a launch.
enum { EVAL_TUPLES = 0, EVAL_ROW = 1, EVAL_COL = 2 };

struct EvalArgs {
  int mode;
  long long n;
  const int* idx;        // EVAL_TUPLES: [n][d]
  const int* pivot;      // EVAL_ROW: device pointer to the row pivot; EVAL_COL: to the column pivot
  const int* done;       // optional device flag: when non-zero the launch does nothing
  const int* skip;       // optional second flag with the same effect
  int nper;              // EVAL_ROW / EVAL_COL with a block of fibres: entries per fibre
                         //   (0: one fibre at *pivot); entry e is element e % nper of the
                         //   fibre at pivot[e / nper]
  const int* nact;       // optional device count of active fibres of the block (entries of
                         //   fibres >= *nact are not evaluated)
  int kterms;            // number of residual terms l < kterms
  const int* kidx;       // optional device iteration index kk: pivot += kk, kterms = kk,
  long long out_stride;  //   out += kk * out_stride (cross-approximation graph)
  const double* X;       // residual out[e] = val - sum_l X[*pivot + l*ldX] * Y[e + l*ldY]
  long long ldX;
  const double* Y;
  long long ldY;
  double* out;           // [n]
  double tau;
  const double* E;       // [dx][NX] frozen field
  const float* E32;      // its FP32 copy (FP32 / BF16x3 paths)
  int foot_euler;
};

// Per-call parameters of the entry evaluator kept in device memory, so that a captured
// CUDA graph serves every SLAR call of a context.
template <typename T>
struct EvalParams {
  HTView<T> ht;
  CorrView corr;
  double tau;
  const double* E;
  const float* E32;
  int foot_euler;
};

// ---- launchers (defined in the .cu files) ----
// `tile` = entries per CTA of the evaluator, 16, 32 or 64 (chosen by the autotuner)
bool eval_tile_ok(int tile);
template <typename T>
cudaError_t launch_sl_eval(const GridDesc& g, const HTView<T>& ht, const CorrView& corr,
                           const EvalArgs& a, int evaluate_at_grid, cudaStream_t s, int tile = 32);
// launch reading HT / field / tau from device memory; smem_bytes fixed by the caller
template <typename T>
cudaError_t launch_sl_eval_dev(const GridDesc& g, const EvalParams<T>* P, const EvalArgs& a,
                               size_t smem_bytes, cudaStream_t s, int tile = 32);
template <typename T>
size_t sl_eval_smem(const GridDesc& g, const int* ranks6, int tile = 32);
// the largest evaluator tile <= tile whose shared memory fits the opt-in limit at these ranks
template <typename T>
int sl_eval_fit_tile(const GridDesc& g, const int* ranks6, int tile);
// opt the evaluator kernels into large dynamic shared memory (call before any capture)
cudaError_t sl_eval_init_attrs();
cudaError_t linalg_init_attrs();
// tensor-core (tcgen05) evaluator for d = 4 trees (sl_eval_tc.cu): a prologue kernel (feet,
// leaf gathers, operand split; several CTAs per SM) writes per-entry scratch that the
// tensor-core kernel (128 entries per CTA, one CTA per SM) reads; pieces = 2 (BF16x3) or 3
// (BF16x6); b12 / b34 are the transfer tensors pre-split by split_transfer_bf16 with the same
// piece count (tc_split_bytes(pieces) each); err (device int) is set if an MMA completion
// wait runs out.  Scratch: tc_scratch_bytes(cap) bytes for cap entries (a multiple of 128).
struct TcScratch {
  unsigned char* a;   // A tiles per 128-entry tile
  float* c1;          // [cap][2][64]
  int* rows;          // [cap][12]
  float* w;           // [cap][12]
  long long cap;
};
long long tc_scratch_bytes(long long cap);
TcScratch tc_scratch_view(void* base, long long cap);
size_t sl_eval_tc_smem(const int* ranks6, int pieces);
long long tc_split_bytes(int pieces);
cudaError_t sl_eval_tc_init_attrs();
cudaError_t split_transfer_bf16(const float* B, int rp, int ra, int rb, void* out, int pieces, cudaStream_t s);
// Broot [r12][r34] pre-split for the root contraction on the tensor cores (<= 24 KiB)
cudaError_t split_root_bf16(const float* Broot, int r12, int r34, void* out, int pieces, cudaStream_t s);
cudaError_t launch_sl_eval_tc(const GridDesc& g, const HTView<float>& ht, const CorrView& corr, const EvalArgs& a,
                              const void* b12, const void* b34, const void* broot, int* err, int pieces,
                              const TcScratch& sc, cudaStream_t s);
cudaError_t launch_sl_eval_tc_dev(const GridDesc& g, const EvalParams<float>* P, const EvalArgs& a, const void* b12,
                                  const void* b34, const void* broot, int* err, int pieces, size_t smem_bytes,
                                  const TcScratch& sc, cudaStream_t s);

// dense FP64 linear algebra (linalg.cu)
// C[b] = alpha op(A[b]) op(B[b]) + beta C[b]; row-major; op(A) is M x K.
cudaError_t dgemm(int tA, int tB, int M, int N, int K, double alpha, const double* A, int lda,
                  long long sA, const double* B, int ldb, long long sB, double beta, double* C,
                  int ldc, long long sC, int batch, cudaStream_t s);
// G = A^T A for A column-major m x n (column stride lda); partial sums over row blocks are
// reduced in a fixed order (deterministic).  work needs nblk*n*n doubles.
cudaError_t gram_tall(const double* A, long long lda, int m, int n, double* G, double* work,
                      int work_blocks, cudaStream_t s);
// out[i][j] = sum_p sum_c X[p][i][c] Y[p][j][c]   (X: P x I x C, Y: P x J x C)
cudaError_t contract_last(const double* X, const double* Y, int P, int I, int J, int C,
                          double* out, double* work, long long work_len, cudaStream_t s);
// out[i][j] = sum_p sum_c X[p][c][i] Y[p][c][j]   (X: P x C x I, Y: P x C x J)
cudaError_t contract_mid(const double* X, const double* Y, int P, int C, int I, int J,
                         double* out, double* work, long long work_len, cudaStream_t s);
// Cholesky of an n x n SPD matrix (row-major), returns upper R (G = R^T R) and R^{-1};
// info[0] != 0 on breakdown.
cudaError_t chol_inv(const double* G, int n, double* R, double* Rinv, int* info, cudaStream_t s);
// Householder QR of a column-major m x n matrix A (destroyed): Q column-major m x n,
// R row-major n x n upper triangular, tau[n] scratch.  One CTA; for set-up paths.
cudaError_t householder_qr(double* A, int m, int n, double* Q, double* R, double* tau,
                           cudaStream_t s);
// Symmetric eigendecomposition of a batch of matrices (cyclic Jacobi, one CTA each).
// A[b]: n_b x n_b row-major (ld = n_b), W[b]: n_b eigenvalues descending,
// V[b]: n_b x n_b eigenvectors as columns (row-major, ld = n_b).
struct EigJob {
  const double* A;
  double* W;
  double* V;
  double* work;  // 2 (SLAR_MAX_N+1)^2 doubles scratch
  int n;
  double floor_rel;     // off-diagonals below floor_rel ||A||_F are not rotated
  double compress_rel;  // > 0: pivoted-Cholesky compression down to compress_rel x trace first
  int nvec;             // leading eigenvectors the caller reads (<= n)
  int tri;              // 1: a compressed rank above 40 goes to the tridiagonal solver, which
                        // returns the nvec leading eigenpairs, W[nvec] = the rest of the trace
                        // and W[i > nvec] = 0
};
cudaError_t eig_batched(const EigJob* jobs_host, int njobs, EigJob* jobs_dev, cudaStream_t s);
// Rank selection from descending eigenvalues: smallest k with tail sum <= thr2, k in [1, cap].
// If that k exceeds cap (the tolerance cannot be met within the cap), *capped (when given)
// is set to 1.
struct RankJob {
  const double* W;
  int n;
  int cap;
  int* out;
  int* capped;
};
cudaError_t choose_ranks(const RankJob* jobs_host, int njobs, RankJob* jobs_dev, const double* normF2,
                         double scale, cudaStream_t s);
cudaError_t transpose(const double* A, int rows, int cols, double* B, cudaStream_t s);  // B = A^T
cudaError_t copy_cols(const double* A, int lda_rows, int rows, int cols, double* B, int ldb,
                      cudaStream_t s);
cudaError_t to_float(const double* a, float* b, long long n, cudaStream_t s);
// up to 8 FP64 -> FP32 conversions in one launch
struct F32Batch {
  const double* a[8];
  float* b[8];
  long long off[9] = {0};
  int k = 0;
  void add(const double* src, float* dst, long long n);
};
cudaError_t to_float_batch(const F32Batch& bt, cudaStream_t s);
cudaError_t fill_identity(double* A, int n, int ld, cudaStream_t s);
cudaError_t fill_zero(double* A, long long n, cudaStream_t s);

}  // namespace slar
