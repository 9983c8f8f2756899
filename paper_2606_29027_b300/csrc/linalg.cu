// Dense FP64 building blocks of the HT truncation (Supp. B.1: orthogonalisation, Gram
// matrices of the dimension-tree nodes, small symmetric eigenproblems) -- all hand-written.
#include "common.cuh"

#include <math.h>
#include <vector>

namespace slar {
namespace {

// ---------------------------------------------------------------------------------------
// strided-batched DGEMM, row-major, 32x32 output tile per CTA, 256 threads x 4 outputs
// ---------------------------------------------------------------------------------------
constexpr int GT = 32;
constexpr int GK = 16;

__global__ void __launch_bounds__(256)
k_dgemm(int tA, int tB, int M, int N, int K, double alpha, const double* __restrict__ A, int lda,
        long long sA, const double* __restrict__ B, int ldb, long long sB, double beta,
        double* __restrict__ C, int ldc, long long sC) {
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const int bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int row0 = blockIdx.y * GT, col0 = blockIdx.x * GT;
  const int tid = threadIdx.x;
  const int tx = tid & 31, ty = tid >> 5;  // ty 0..7 -> rows ty, ty+8, ty+16, ty+24
  double acc[4] = {0, 0, 0, 0};
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int it = tid; it < GK * GT; it += 256) {
      int kk, mm;
      if (tA) { mm = it % GT; kk = it / GT; } else { kk = it % GK; mm = it / GK; }
      const int gm = row0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gm < M && gk < K) v = tA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
      As[kk][mm] = v;
    }
    for (int it = tid; it < GK * GT; it += 256) {
      int kk, nn;
      if (tB) { kk = it % GK; nn = it / GK; } else { nn = it % GT; kk = it / GT; }
      const int gn = col0 + nn, gk = k0 + kk;
      double v = 0.0;
      if (gn < N && gk < K) v = tB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      const double b = Bs[kk][tx];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i] += As[kk][ty + 8 * i] * b;
    }
    __syncthreads();
  }
  const int gn = col0 + tx;
  if (gn < N) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gm = row0 + ty + 8 * i;
      if (gm < M) {
        double* c = C + (long long)gm * ldc + gn;
        *c = alpha * acc[i] + (beta == 0.0 ? 0.0 : beta * *c);
      }
    }
  }
}

// Small-output variant: T x T output tile per CTA, one output per thread.  The truncation's
// GEMMs are mostly 64 x 64 or smaller: 32 x 32 tiles leave four CTAs on a GPU whose FP64
// rate per SM is low, so smaller tiles spread the same work over 4-16 times more SMs.
template <int T>
__global__ void __launch_bounds__(T * T)
k_dgemm_small(int tA, int tB, int M, int N, int K, double alpha, const double* __restrict__ A, int lda,
              long long sA, const double* __restrict__ B, int ldb, long long sB, double beta,
              double* __restrict__ C, int ldc, long long sC) {
  __shared__ double As[GK][T + 1];
  __shared__ double Bs[GK][T + 1];
  const int bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int row0 = blockIdx.y * T, col0 = blockIdx.x * T;
  const int tid = threadIdx.x;
  const int tx = tid % T, ty = tid / T;
  double acc = 0.0;
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int it = tid; it < GK * T; it += T * T) {
      int kk, mm;
      if (tA) { mm = it % T; kk = it / T; } else { kk = it % GK; mm = it / GK; }
      const int gm = row0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gm < M && gk < K) v = tA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
      As[kk][mm] = v;
    }
    for (int it = tid; it < GK * T; it += T * T) {
      int kk, nn;
      if (tB) { kk = it % GK; nn = it / GK; } else { nn = it % T; kk = it / T; }
      const int gn = col0 + nn, gk = k0 + kk;
      double v = 0.0;
      if (gn < N && gk < K) v = tB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) acc += As[kk][ty] * Bs[kk][tx];
    __syncthreads();
  }
  const int gm = row0 + ty, gn = col0 + tx;
  if (gm < M && gn < N) {
    double* c = C + (long long)gm * ldc + gn;
    *c = alpha * acc + (beta == 0.0 ? 0.0 : beta * *c);
  }
}

// ---------------------------------------------------------------------------------------
// G = A^T A for a tall column-major A (m x n, n <= 64): each CTA reduces ROWS rows into a
// partial n x n; a second kernel sums the partials in block order.  (Summing them in the CTA
// that finishes last instead puts n^2 chains of nblk dependent L2 loads on one SM, which costs
// more on B300 than the second launch.)
// ---------------------------------------------------------------------------------------
constexpr int GR_ROWS = 64;

__global__ void __launch_bounds__(256)
k_gram_partial(const double* __restrict__ A, long long lda, int m, int n, double* __restrict__ part) {
  __shared__ double tile[GR_ROWS][SLAR_MAX_RANK + 1];
  const int r0 = blockIdx.x * GR_ROWS;
  const int rows = min(GR_ROWS, m - r0);
  for (int it = threadIdx.x; it < GR_ROWS * n; it += 256) {
    const int c = it / GR_ROWS, rr = it % GR_ROWS;
    tile[rr][c] = (rr < rows) ? A[(long long)c * lda + r0 + rr] : 0.0;
  }
  __syncthreads();
  double* out = part + (long long)blockIdx.x * n * n;
  for (int it = threadIdx.x; it < n * n; it += 256) {
    const int i = it / n, j = it % n;
    double s = 0.0;
    for (int rr = 0; rr < rows; ++rr) s += tile[rr][i] * tile[rr][j];
    out[it] = s;
  }
}

__global__ void k_sum_partials(const double* __restrict__ part, int nblk, int nn, double* __restrict__ G) {
  const int it = blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= nn) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(long long)b * nn + it];
  G[it] = s;
}

// out[i][j] = sum_p sum_c X(p, i, c) Y(p, j, c) with general strides; a CTA computes a
// 16 x 16 output tile over one p-group and writes a partial; partials are summed in group
// order (deterministic).
constexpr int CT = 16;
constexpr int CK = 16;

__global__ void __launch_bounds__(256)
k_contract(const double* __restrict__ X, long long xp, long long xi, long long xc,
           const double* __restrict__ Y, long long yp, long long yj, long long yc, int P, int I,
           int J, int C, int pgroup, double* __restrict__ part) {
  __shared__ double xs[CK][CT + 1], ys[CK][CT + 1];
  const int ti = threadIdx.x / CT, tj = threadIdx.x % CT;
  const int i0 = blockIdx.y * CT, j0 = blockIdx.x * CT;
  const int g = blockIdx.z;
  const int p0 = g * pgroup, p1 = min(P, p0 + pgroup);
  double acc = 0.0;
  for (int p = p0; p < p1; ++p) {
    for (int c0 = 0; c0 < C; c0 += CK) {
      for (int it = threadIdx.x; it < CK * CT; it += 256) {
        const int cc = it % CK, r = it / CK;
        const int c = c0 + cc;
        xs[cc][r] = (c < C && i0 + r < I) ? X[p * xp + (long long)(i0 + r) * xi + c * xc] : 0.0;
        ys[cc][r] = (c < C && j0 + r < J) ? Y[p * yp + (long long)(j0 + r) * yj + c * yc] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int cc = 0; cc < CK; ++cc) acc += xs[cc][ti] * ys[cc][tj];
      __syncthreads();
    }
  }
  if (i0 + ti < I && j0 + tj < J) part[((long long)g * I + i0 + ti) * J + j0 + tj] = acc;
}

// ---------------------------------------------------------------------------------------
// Cholesky G = R^T R (R upper) and R^{-1}, one CTA, n <= 64.
// ---------------------------------------------------------------------------------------
__global__ void k_chol_inv(const double* __restrict__ G, int n, double* __restrict__ R,
                           double* __restrict__ Rinv, int* info) {
  // Column-equilibrated: factor D^{-1} G D^{-1} = Rt^T Rt with D = diag(sqrt(G_ii)), then
  // R = Rt D and R^{-1} = D^{-1} Rt^{-1}.  Equilibration makes the factorisation
  // insensitive to the column scaling of the matrix whose Gram G is.  B300 retires FP64 at a
  // low rate with a long latency, so every division is taken once (reciprocals of the scale
  // factors and of the pivots) and the chains use multiplications.
  extern __shared__ double chol_smem[];
  double (*a)[SLAR_MAX_RANK + 1] = reinterpret_cast<double (*)[SLAR_MAX_RANK + 1]>(chol_smem);
  double (*ri)[SLAR_MAX_RANK + 1] =
      reinterpret_cast<double (*)[SLAR_MAX_RANK + 1]>(chol_smem + SLAR_MAX_RANK * (SLAR_MAX_RANK + 1));
  __shared__ double dsc[SLAR_MAX_RANK], dinv[SLAR_MAX_RANK], rinv[SLAR_MAX_RANK];
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  for (int i = tid; i < n; i += blockDim.x) {
    const double gii = G[i * n + i];
    dsc[i] = gii > 0.0 ? sqrt(gii) : 1.0;
    dinv[i] = 1.0 / dsc[i];
  }
  __syncthreads();
  for (int it = tid; it < n * n; it += blockDim.x) {
    const int i = it / n, j = it % n;
    a[i][j] = G[it] * dinv[i] * dinv[j];
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      const double dkk = a[k][k];
      double rkk;
      if (!(dkk > 0.0)) { bad = k + 1; rkk = 1.0; }
      else rkk = sqrt(dkk);
      a[k][k] = rkk;
      rinv[k] = 1.0 / rkk;
    }
    __syncthreads();
    const double rk = rinv[k];
    for (int j = k + 1 + tid; j < n; j += blockDim.x) a[k][j] *= rk;
    __syncthreads();
    for (int it = tid; it < (n - k - 1) * (n - k - 1); it += blockDim.x) {
      const int i = k + 1 + it / (n - k - 1), j = k + 1 + it % (n - k - 1);
      if (j >= i) a[i][j] -= a[k][i] * a[k][j];
    }
    __syncthreads();
  }
  // R^{-1} column by column (back substitution, one column per thread)
  for (int j = tid; j < n; j += blockDim.x) {
    for (int i = 0; i < n; ++i) ri[i][j] = 0.0;
    ri[j][j] = rinv[j];
    for (int i = j - 1; i >= 0; --i) {
      double s = 0.0;
      for (int k2 = i + 1; k2 <= j; ++k2) s += a[i][k2] * ri[k2][j];
      ri[i][j] = -s * rinv[i];
    }
  }
  __syncthreads();
  for (int it = tid; it < n * n; it += blockDim.x) {
    const int i = it / n, j = it % n;
    R[it] = (j >= i) ? a[i][j] * dsc[j] : 0.0;
    Rinv[it] = ri[i][j] * dinv[i];
  }
  if (tid == 0 && bad) info[0] = bad;
}

// ---------------------------------------------------------------------------------------
// Householder QR of a column-major m x n matrix (n <= 64, m >= n) held in global memory,
// one CTA.  Robust to rank deficiency (Q stays orthonormal).  A is overwritten by the
// reflectors; Q (column-major m x n, ld m) and R (row-major n x n) are written out.
// ---------------------------------------------------------------------------------------
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  const int nw = blockDim.x >> 5;
  for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

__global__ void __launch_bounds__(256)
k_householder(double* A, int m, int n, double* Q, double* R, double* tau) {
  __shared__ double red[8];
  const int tid = threadIdx.x;
  for (int j = 0; j < n; ++j) {
    double* x = A + (long long)j * m;
    double ss = 0.0;
    for (int i = j + tid; i < m; i += 256) ss += x[i] * x[i];
    const double nrm2 = block_sum(ss, red);
    const double x0 = x[j];
    const double nrm = sqrt(nrm2);
    double alpha = (x0 >= 0.0) ? -nrm : nrm;
    double t = 0.0;
    __syncthreads();
    if (nrm > 0.0) {
      // v = x - alpha e_j (stored in x[j:]), tau = 2 / (v^T v)
      const double v0 = x0 - alpha;
      const double vv = nrm2 - x0 * x0 + v0 * v0;
      t = vv > 0.0 ? 2.0 / vv : 0.0;
      if (tid == 0) x[j] = v0;
    } else {
      alpha = 0.0;
    }
    __syncthreads();
    if (tid == 0) { tau[j] = t; R[j * n + j] = alpha; }
    for (int k = j + 1; k < n; ++k) {
      double* y = A + (long long)k * m;
      double dp = 0.0;
      for (int i = j + tid; i < m; i += 256) dp += x[i] * y[i];
      const double s = block_sum(dp, red) * t;
      for (int i = j + tid; i < m; i += 256) y[i] -= s * x[i];
      __syncthreads();
      if (tid == 0) R[j * n + k] = y[j];
    }
    __syncthreads();
    if (tid == 0) for (int k = 0; k < j; ++k) R[j * n + k] = 0.0;
  }
  // Q = H_0 ... H_{n-1} [I; 0], accumulated backwards
  for (int it = tid; it < m * n; it += 256) {
    const int c = it / m, i = it % m;
    Q[it] = (i == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = n - 1; j >= 0; --j) {
    const double* x = A + (long long)j * m;
    const double t = tau[j];
    for (int c = j; c < n; ++c) {
      double* q = Q + (long long)c * m;
      double dp = 0.0;
      for (int i = j + tid; i < m; i += 256) dp += x[i] * q[i];
      const double s = block_sum(dp, red) * t;
      for (int i = j + tid; i < m; i += 256) q[i] -= s * x[i];
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------------------
// Cyclic Jacobi eigensolver, one CTA per matrix (n <= 128).  Round-robin ordering: in each
// round n/2 disjoint rotations are applied at once as 2x2 block updates A <- J^T A J,
// V <- V J.  The matrix lives in shared memory, the eigenvectors in global scratch.
// ---------------------------------------------------------------------------------------
constexpr int EIG_THREADS = 512;

// Cyclic Jacobi sweeps on the ne x ne symmetric matrix sA (shared memory) accumulating
// eigenvectors in V (global, ne x ne).  Round-robin ordering: each round applies ne/2
// disjoint rotations at once as 2x2 block updates A <- J^T A J, V <- V J.  A pair is
// rotated while |a_pq| > tol sqrt(|a_pp a_qq|) (relative criterion: small eigenvalues and
// their eigenvectors are resolved to relative accuracy); stop after a sweep without any
// rotation, or after 40 sweeps.  Entries below floor_rel ||A||_F are never rotated: 1e-17 for
// Gram matrices of FP64 data (the rounding level), 1e-13 for those of FP32 entries and 1e-9
// for BF16x3 entries, whose noise puts a cluster of eigenvalues near u^2 ||A|| (u the
// entries' relative precision) that carries no information.
template <int NT>
__device__ void jacobi_sweeps(double* sA, int ne, double* V, int* pp, int* qq, double* cc,
                              double* ss, int* rotated, double floor_rel) {
  const int tid = threadIdx.x;
  const int half = ne / 2;
  const int m = ne - 1;
  const double tol = 1e-15;
  __shared__ unsigned short tri[(SLAR_MAX_N / 2) * (SLAR_MAX_N / 2 + 1) / 2];
  __shared__ double fro_red[NT / 32];
  __shared__ double floor_s;
  // absolute floor: entries at the rounding (or data-noise) level of the matrix are not rotated
  {
    double f = 0.0;
    for (int it = tid; it < ne * ne; it += NT) f += sA[it] * sA[it];
    for (int o = 16; o > 0; o >>= 1) f += __shfl_down_sync(0xffffffffu, f, o);
    if ((tid & 31) == 0) fro_red[tid >> 5] = f;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < NT / 32; ++w) t += fro_red[w];
      floor_s = floor_rel * sqrt(t);
    }
    __syncthreads();
  }
  const double afloor = floor_s;
  for (int ia = tid; ia < half; ia += NT) {
    const int off = ia * half - ia * (ia - 1) / 2;
    for (int ib = ia; ib < half; ++ib) tri[off + ib - ia] = (unsigned short)((ia << 8) | ib);
  }
  __syncthreads();
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (tid == 0) *rotated = 0;
    __syncthreads();
    for (int rnd = 0; rnd < m; ++rnd) {
      for (int k = tid; k < half; k += NT) {
        int p, q;
        if (k == 0) { p = rnd; q = ne - 1; }
        else { p = (rnd + k) % m; q = (rnd - k + m) % m; }
        if (p > q) { const int t = p; p = q; q = t; }
        const double apq = sA[p * ne + q];
        const double app = sA[p * ne + p], aqq = sA[q * ne + q];
        double c = 1.0, s = 0.0;
        // On B300 a dependent FP64 division costs ~440 cycles and a square root ~680, so the
        // test is squared and the angle is taken in FP32:
        //   theta = d / e (d = a_qq - a_pp, e = 2 a_pq),
        //   t = sgn(theta) / (|theta| + sqrt(theta^2 + 1)) = sgn(d e) |e| / (|d| + sqrt(d^2 + e^2)),
        //   c = 1 / sqrt(t^2 + 1), s = t c,
        // from d and e scaled by the same power of two (exact); (c, s) is then made orthonormal
        // to FP64 precision by two Newton steps for 1 / sqrt(c^2 + s^2) (FMAs only).  Any
        // exactly orthogonal rotation keeps the spectrum; an angle good to 2^-24 leaves
        // a'_pq ~ 1e-7 a_pq, which the sweeps clear like any other off-diagonal entry, and the
        // stop test stays in FP64.
        if (apq * apq > tol * tol * fabs(app * aqq) && fabs(apq) > afloor) {
          const double d = aqq - app, e = 2.0 * apq;
          int ex;
          frexp(fmax(fabs(d), fabs(e)), &ex);
          const float df = (float)ldexp(d, -ex), ef = (float)ldexp(e, -ex);
          const float tf = (df * ef >= 0.f ? 1.f : -1.f) * fabsf(ef) / (fabsf(df) + sqrtf(df * df + ef * ef));
          const float cf = rsqrtf(fmaf(tf, tf, 1.f));
          c = (double)cf;
          s = (double)(tf * cf);
#pragma unroll
          for (int it = 0; it < 2; ++it) {
            const double r = fma(c, c, s * s);
            const double kf = fma(-0.5, r, 1.5);
            c *= kf;
            s *= kf;
          }
          *rotated = 1;
        }
        pp[k] = p; qq[k] = q; cc[k] = c; ss[k] = s;
      }
      __syncthreads();
      // upper-triangular block pairs (ia <= ib) from the precomputed table; the
      // transposed block is mirrored
      const int nblk = half * (half + 1) / 2;
      for (int it = tid; it < nblk; it += NT) {
        const int ia = tri[it] >> 8, ib = tri[it] & 0xff;
        const double sa = ss[ia], sb = ss[ib];
        if (sa == 0.0 && sb == 0.0) continue;
        const int pa = pp[ia], qa = qq[ia], pb = pp[ib], qb = qq[ib];
        const double ca = cc[ia], cb = cc[ib];
        const double x00 = sA[pa * ne + pb], x01 = sA[pa * ne + qb];
        const double x10 = sA[qa * ne + pb], x11 = sA[qa * ne + qb];
        // J^T X : rows (p, q) -> (c x_p - s x_q, s x_p + c x_q); then (.) J on columns
        const double y00 = ca * x00 - sa * x10, y01 = ca * x01 - sa * x11;
        const double y10 = sa * x00 + ca * x10, y11 = sa * x01 + ca * x11;
        const double z00 = cb * y00 - sb * y01, z01 = sb * y00 + cb * y01;
        const double z10 = cb * y10 - sb * y11, z11 = sb * y10 + cb * y11;
        sA[pa * ne + pb] = z00;
        sA[pa * ne + qb] = z01;
        sA[qa * ne + pb] = z10;
        sA[qa * ne + qb] = z11;
        if (ia != ib) {
          sA[pb * ne + pa] = z00;
          sA[qb * ne + pa] = z01;
          sA[pb * ne + qa] = z10;
          sA[qb * ne + qa] = z11;
        }
      }
      for (int it = tid; it < ne * half; it += NT) {
        const int row = it / half, ib = it % half;
        const double sb = ss[ib];
        if (sb == 0.0) continue;
        const int pb = pp[ib], qb = qq[ib];
        const double cb = cc[ib];
        const double vp = V[row * ne + pb], vq = V[row * ne + qb];
        V[row * ne + pb] = cb * vp - sb * vq;
        V[row * ne + qb] = sb * vp + cb * vq;
      }
      __syncthreads();
    }
    if (!*rotated) break;
    __syncthreads();
  }
}

// Symmetric eigendecomposition, one CTA per matrix.  Matrices with n > 24 are first
// compressed by a pivoted Cholesky factorisation G = L L^T stopped at the numerical rank
// (remaining diagonal <= 1e-16 trace); the eigenpairs of the small M = L^T L give those of
// G: lambda(G) = lambda(M), S = L V Lambda^{-1/2}.  Eigenvalues beyond the numerical rank
// are returned as 0 with zero eigenvectors.  L, M and the Jacobi eigenvectors stay in
// shared memory; only a full-rank matrix with n > 64 falls back to eigenvectors in global
// memory.
constexpr int EIG_RTMAX = 64;
constexpr int TRI_RT = 40;                                          // see EigJob::tri
constexpr int TRI_WORK = 2 * (SLAR_MAX_N + 1) * (SLAR_MAX_N + 1);    // doubles of EigJob::work
constexpr int TRI_FLAG = TRI_WORK - 1;                              // 1.0: job handed over
constexpr int TRI_TRACE = TRI_WORK - 2;                             // trace of the matrix
constexpr int EIG_SMEM_DOUBLES = SLAR_MAX_N * EIG_RTMAX + 2 * EIG_RTMAX * EIG_RTMAX + SLAR_MAX_N;

template <int NT>
__device__ void sort_write(const double* sA, int ne, int n, const double* V, int ldv, double* W,
                           double* Vout) {
  for (int i = threadIdx.x; i < n; i += NT) {
    const double li = sA[i * ne + i];
    int pos = 0;
    for (int j = 0; j < n; ++j) {
      const double lj = sA[j * ne + j];
      pos += (lj > li) || (lj == li && j < i);
    }
    W[pos] = li;
    for (int r = 0; r < n; ++r) Vout[r * n + pos] = V[r * ldv + i];
  }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_jacobi(EigJob* jobs, long long smem_doubles) {
  extern __shared__ double smem[];
  __shared__ int pp[SLAR_MAX_N / 2], qq[SLAR_MAX_N / 2];
  __shared__ double cc[SLAR_MAX_N / 2], ss[SLAR_MAX_N / 2];
  __shared__ double wred[NT / 32];
  __shared__ int wred_i[NT / 32];
  __shared__ int piv_s, rotated, rt_s;
  __shared__ double dpiv_s, dinv_s, trace_s;
  const EigJob job = jobs[blockIdx.x];
  const int n = job.n;
  const int tid = threadIdx.x;
  if (job.compress_rel > 0.0 && n > 24) {
    double* L = smem;                                   // n x rt, column j at L + j n
    double* M = smem + SLAR_MAX_N * EIG_RTMAX;          // ne x ne
    double* Vs = M + EIG_RTMAX * EIG_RTMAX;             // ne x ne
    double* dg = Vs + EIG_RTMAX * EIG_RTMAX;            // n
    for (int i = tid; i < n; i += NT) dg[i] = job.A[i * n + i];
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int i = 0; i < n; ++i) t += fmax(dg[i], 0.0);
      trace_s = t;
      rt_s = 0;
    }
    __syncthreads();
    // stop once the trace left outside L L^T is at most compress_rel x trace: the eigenvalues
    // dropped with it lie far below the rank threshold of the truncation
    const double stop = job.compress_rel * trace_s;
    const int rcap = job.tri ? TRI_RT + 1 : EIG_RTMAX;
    const int rtmax = n < rcap ? n : rcap;
    // the reductions run on the warps that hold entries only: FP64 compares and adds of idle
    // warps would queue on the SM's FP64 units like real work
    const int nwa = (n + 31) / 32 < NT / 32 ? (n + 31) / 32 : NT / 32;
    const bool act = (tid >> 5) < nwa;
    for (int j = 0; j < rtmax; ++j) {
      double best = -1.0;
      int bi = -1;
      if (act) {
        for (int i = tid; i < n; i += NT)
          if (dg[i] > best) { best = dg[i]; bi = i; }
        for (int o = 16; o > 0; o >>= 1) {
          const double ob = __shfl_down_sync(0xffffffffu, best, o);
          const int oi = __shfl_down_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi >= 0 && (bi < 0 || oi < bi))) { best = ob; bi = oi; }
        }
        if ((tid & 31) == 0) { wred[tid >> 5] = best; wred_i[tid >> 5] = bi; }
      }
      __syncthreads();
      if (tid == 0) {
        double b = -1.0;
        int ib = -1;
        for (int w = 0; w < nwa; ++w)
          if (wred[w] > b || (wred[w] == b && wred_i[w] >= 0 && (ib < 0 || wred_i[w] < ib))) {
            b = wred[w]; ib = wred_i[w];
          }
        piv_s = ib;
        dpiv_s = b;
        // one reciprocal square root for the CTA: on B300 an FP64 sqrt and division cost
        // tens of FP64-pipe instructions, and every warp computing them serialises on the
        // SM's few FP64 units
        dinv_s = b > 0.0 ? 1.0 / sqrt(b) : 0.0;
      }
      __syncthreads();
      if (!(dpiv_s > 0.0) || piv_s < 0) break;
      const int p = piv_s;
      const double inv = dinv_s;
      double* lj = L + j * n;
      for (int i = tid; i < n; i += NT) {
        double v = job.A[i * n + p];
        for (int t = 0; t < j; ++t) v -= L[t * n + i] * L[t * n + p];
        lj[i] = v * inv;
      }
      __syncthreads();
      if (act) {
        double rem = 0.0;
        for (int i = tid; i < n; i += NT) {
          const double v = (i == p) ? -1.0 : dg[i] - lj[i] * lj[i];
          dg[i] = v;
          rem += fmax(v, 0.0);
        }
        for (int o = 16; o > 0; o >>= 1) rem += __shfl_down_sync(0xffffffffu, rem, o);
        if ((tid & 31) == 0) wred[tid >> 5] = rem;
      }
      __syncthreads();
      if (tid == 0) {
        rt_s = j + 1;
        double t = 0.0;
        for (int w = 0; w < nwa; ++w) t += wred[w];
        dpiv_s = t;   // trace left outside L L^T
      }
      __syncthreads();
      if (!(dpiv_s > stop)) break;
    }
    int rt = rt_s;
    const bool full = (rt == rtmax && rtmax < n && dpiv_s > stop);
    if (job.tri) {
      // numerical rank above TRI_RT: the FP64 Jacobi of the compressed matrix would cost
      // O(rt^3) per sweep on one SM; the tridiagonal solver takes the job instead
      const bool hand_off = full || rt > TRI_RT;
      if (tid == 0) {
        job.work[TRI_FLAG] = hand_off ? 1.0 : 0.0;
        job.work[TRI_TRACE] = trace_s;
      }
      if (hand_off) return;
    }
    if (!full) {
      if (rt == 0) {  // zero matrix: one zero eigenpair
        rt = 1;
        for (int i = tid; i < n; i += NT) L[i] = 0.0;
      }
      const int ne = rt + (rt & 1);
      __syncthreads();
      for (int it = tid; it < ne * ne; it += NT) {
        const int a = it / ne, b = it % ne;
        double v = 0.0;
        if (a < rt && b < rt)
          for (int i = 0; i < n; ++i) v += L[a * n + i] * L[b * n + i];
        M[it] = v;
        Vs[it] = (a == b) ? 1.0 : 0.0;
      }
      __syncthreads();
      jacobi_sweeps<NT>(M, ne, Vs, pp, qq, cc, ss, &rotated, job.floor_rel);
      // eigenvalue order of M (descending, ties by index); 1/sqrt(lambda) once per eigenvalue
      __shared__ int order[EIG_RTMAX];
      __shared__ double isq[EIG_RTMAX];
      for (int i = tid; i < rt; i += NT) {
        const double li = M[i * ne + i];
        int pos = 0;
        for (int j = 0; j < rt; ++j) {
          const double lj = M[j * ne + j];
          pos += (lj > li) || (lj == li && j < i);
        }
        order[pos] = i;
        job.W[pos] = li > 0.0 ? li : 0.0;
        isq[pos] = li > 0.0 ? 1.0 / sqrt(li) : 0.0;
      }
      for (int i = rt + tid; i < n; i += NT) job.W[i] = 0.0;
      __syncthreads();
      // S[r][pos] = sum_a L[r][a] V[a][i] / sqrt(lambda_i)
      for (int it = tid; it < n * n; it += NT) {
        const int r = it / n, pos = it % n;
        double v = 0.0;
        if (pos < rt) {
          const int i = order[pos];
          const double is = isq[pos];
          if (is > 0.0) {
            for (int a = 0; a < rt; ++a) v += L[a * n + r] * Vs[a * ne + i];
            v *= is;
          }
        }
        job.V[it] = v;
      }
      return;
    }
    __syncthreads();
    // full-rank large matrix: direct Jacobi with eigenvectors in global scratch
    const int ne = n + (n & 1);
    double* sA = smem;
    double* V = job.work;
    for (int it = tid; it < ne * ne; it += NT) {
      const int i = it / ne, j = it % ne;
      sA[it] = (i < n && j < n) ? job.A[i * n + j] : 0.0;
      V[it] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    jacobi_sweeps<NT>(sA, ne, V, pp, qq, cc, ss, &rotated, job.floor_rel);
    sort_write<NT>(sA, ne, n, V, ne, job.W, job.V);
    return;
  }
  // the matrix in shared memory; its eigenvectors there too while both fit in the dynamic
  // allocation (smem_doubles), else in the job's global scratch (n > 90)
  const int ne = n + (n & 1);
  double* sA = smem;
  double* V = (2LL * ne * ne <= smem_doubles) ? smem + ne * ne : job.work;
  for (int it = tid; it < ne * ne; it += NT) {
    const int i = it / ne, j = it % ne;
    sA[it] = (i < n && j < n) ? job.A[i * n + j] : 0.0;
    V[it] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  jacobi_sweeps<NT>(sA, ne, V, pp, qq, cc, ss, &rotated, job.floor_rel);
  sort_write<NT>(sA, ne, n, V, ne, job.W, job.V);
}

// ---------------------------------------------------------------------------------------
// Tridiagonal symmetric eigensolver for the jobs k_jacobi hands over (numerical rank above
// TRI_RT of FP32 / BF16x3 data).  On B300 an SM retires about two FP64 FMAs per clock, so a
// cyclic Jacobi of order 64-128 (O(n^3) work per sweep, 6-10 sweeps) takes milliseconds to
// tens of milliseconds on one SM; this path does O(n^3) work once and only for the
// eigenvectors the truncation reads:
//   1. Householder reduction A = Q T Q^T in shared memory (one CTA per matrix);
//   2. the nvec largest eigenvalues of T by multisection on Sturm counts (8 lanes each);
//   3. their eigenvectors of T by inverse iteration (LU with partial pivoting of T - lambda I,
//      three solves from a hashed start vector; one thread each);
//   4. classical Gram-Schmidt applied twice (near-degenerate eigenvalues give non-orthogonal
//      inverse-iteration vectors), then the back-transformation Q z (8 vectors per CTA).
// Eigenvalues are accurate to about u ||A|| (the rank threshold of the truncation is
// eps^2/(2d - 3) ||A|| with eps >= 1e-8, far above).  Outputs follow EigJob::tri.
// Work layout (doubles): [0, n^2) Householder vectors (v_k in row k, entries k+1..n-1), then
// tau[n], d[n], e[n], lambda[n] (descending), Z[nvec][n].
// ---------------------------------------------------------------------------------------
constexpr int TRI_THREADS = 512;
constexpr int TRI_EIG_PER_CTA = 8;

__device__ __forceinline__ bool tri_active(const EigJob& job) {
  return job.tri && job.work[TRI_FLAG] != 0.0;
}

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}

__global__ void __launch_bounds__(TRI_THREADS) k_tri_reduce(const EigJob* jobs) {
  extern __shared__ double sA[];
  __shared__ double sp[SLAR_MAX_N];
  __shared__ double red[TRI_THREADS / 32];
  __shared__ double s_tau;
  const EigJob job = jobs[blockIdx.x];
  if (!tri_active(job)) return;
  const int n = job.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = TRI_THREADS / 32;
  double* wk = job.work;
  double* tau = wk + n * n;
  double* dg = tau + n;
  double* ed = dg + n;
  for (int it = tid; it < n * n; it += TRI_THREADS) sA[it] = job.A[it];
  __syncthreads();
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    double* x = sA + k * n + k + 1;   // row k beyond the diagonal = column k below it
    double ss = 0.0;
    for (int i = 1 + tid; i < m; i += TRI_THREADS) ss += x[i] * x[i];
    const double sigma = block_sum(ss, red);
    if (tid == 0) {
      // H = I - t v v^T with v = x - beta e_1, H x = beta e_1 (beta of sign opposite to x_0)
      const double x0 = x[0];
      double t = 0.0, beta = x0;
      if (sigma > 0.0) {
        const double alpha = sqrt(x0 * x0 + sigma);
        beta = x0 >= 0.0 ? -alpha : alpha;
        const double v0 = x0 - beta;
        t = 2.0 / (sigma + v0 * v0);
        x[0] = v0;
      }
      s_tau = t;
      tau[k] = t;
      dg[k] = sA[k * n + k];
      ed[k] = beta;
    }
    __syncthreads();
    const double t = s_tau;
    for (int i = k + 1 + tid; i < n; i += TRI_THREADS) wk[k * n + i] = sA[k * n + i];
    if (t == 0.0) continue;
    // p = t A' v (a warp per row), w = p - (t/2)(p.v) v, A' <- A' - v w^T - w v^T
    for (int i = k + 1 + warp; i < n; i += NW) {
      double acc = 0.0;
      for (int j = k + 1 + lane; j < n; j += 32) acc += sA[i * n + j] * sA[k * n + j];
      acc = warp_sum_d(acc);
      if (lane == 0) sp[i] = t * acc;
    }
    __syncthreads();
    double pv = 0.0;
    for (int i = k + 1 + tid; i < n; i += TRI_THREADS) pv += sp[i] * sA[k * n + i];
    const double K = 0.5 * t * block_sum(pv, red);
    for (int i = k + 1 + tid; i < n; i += TRI_THREADS) sp[i] -= K * sA[k * n + i];
    __syncthreads();
    for (int i = k + 1 + warp; i < n; i += NW) {
      const double vi = sA[k * n + i], wi = sp[i];
      for (int j = k + 1 + lane; j < n; j += 32) sA[i * n + j] -= vi * sp[j] + wi * sA[k * n + j];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      dg[n - 2] = sA[(n - 2) * n + n - 2];
      ed[n - 2] = sA[(n - 2) * n + n - 1];
      tau[n - 2] = 0.0;
    }
    dg[n - 1] = sA[(n - 1) * n + n - 1];
    tau[n - 1] = 0.0;
  }
}

// Gershgorin interval of T and the pivot floor of the Sturm recurrence
__device__ void tri_bounds(const double* d, const double* e, int n, double* gl, double* gu, double* pivmin) {
  double lo = 1e300, hi = -1e300, e2max = 0.0;
  for (int j = 0; j < n; ++j) {
    const double r = (j > 0 ? fabs(e[j - 1]) : 0.0) + (j + 1 < n ? fabs(e[j]) : 0.0);
    lo = fmin(lo, d[j] - r);
    hi = fmax(hi, d[j] + r);
    if (j + 1 < n) e2max = fmax(e2max, e[j] * e[j]);
  }
  const double bn = fmax(fabs(lo), fabs(hi));
  *pivmin = 2.2250738585072014e-308 * fmax(1.0, e2max);
  *gl = lo - 2.220446049250313e-16 * bn * n - *pivmin;
  *gu = hi + 2.220446049250313e-16 * bn * n + *pivmin;
}

// number of eigenvalues of T below x (Sturm sequence of the LDL^T factorisation of T - x I)
__device__ __forceinline__ int sturm_count(const double* d, const double* e2, int n, double x, double pivmin) {
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  int c = q < 0.0;
  for (int j = 1; j < n; ++j) {
    q = (d[j] - x) - e2[j - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    c += q < 0.0;
  }
  return c;
}

// The nvec largest eigenvalues by multisection: 8 lanes per eigenvalue count the eigenvalues
// below 8 interior points of its interval, and the first point whose count exceeds the
// eigenvalue's index bounds the next interval (9 subintervals per pass: 20 passes shrink the
// Gershgorin interval by 9^20 > 2^63, below the rounding level).  Four eigenvalues per warp,
// one warp per CTA: the dependent Sturm recurrences are latency-bound, so they are spread over
// as many SMs as there are eigenvalue groups.
constexpr int MS_LANES = 8;
constexpr int MS_PASSES = 20;

__global__ void __launch_bounds__(32) k_tri_bisect(const EigJob* jobs) {
  __shared__ double sd[SLAR_MAX_N], se[SLAR_MAX_N], se2[SLAR_MAX_N];
  const EigJob job = jobs[blockIdx.y];
  if (!tri_active(job)) return;
  const int n = job.n;
  const double* wk = job.work;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    sd[j] = wk[n * n + n + j];
    se[j] = j + 1 < n ? wk[n * n + 2 * n + j] : 0.0;
    se2[j] = se[j] * se[j];
  }
  __syncthreads();
  const int grp = threadIdx.x / MS_LANES, l = threadIdx.x % MS_LANES;
  const int tp = blockIdx.x * (32 / MS_LANES) + grp;      // rank from the largest
  const bool valid = tp < job.nvec;
  const int i = n - 1 - (valid ? tp : 0);                 // ascending index
  double lo, hi, pivmin;
  tri_bounds(sd, se, n, &lo, &hi, &pivmin);
  for (int pass = 0; pass < MS_PASSES; ++pass) {
    const double w = (hi - lo) / (double)(MS_LANES + 1);
    const int c = sturm_count(sd, se2, n, lo + (l + 1) * w, pivmin);
    const unsigned above = (__ballot_sync(0xffffffffu, c > i) >> (grp * MS_LANES)) & ((1u << MS_LANES) - 1);
    const int first = above ? __ffs(above) - 1 : MS_LANES;   // first point with lambda_i below it
    const double nlo = first == 0 ? lo : lo + first * w;
    const double nhi = first == MS_LANES ? hi : lo + (first + 1) * w;
    lo = nlo;
    hi = nhi;
  }
  if (valid && l == 0) job.work[n * n + 3 * n + tp] = 0.5 * (lo + hi);
}

__device__ __forceinline__ double hash_unit(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 1.1102230246251565e-16 - 0.5;
}

// inverse iteration on T for the eigenvalue of rank tp: Gaussian elimination with partial
// pivoting of T - lambda I (two superdiagonals of fill), zero pivots replaced by `tiny`
__global__ void k_tri_vec(const EigJob* jobs) {
  const EigJob job = jobs[blockIdx.y];
  if (!tri_active(job)) return;
  const int n = job.n;
  const int tp = blockIdx.x * blockDim.x + threadIdx.x;
  if (tp >= job.nvec) return;
  double* wk = job.work;
  const double* d = wk + n * n + n;
  const double* e = d + n;
  const double* lam = e + n;
  double* z = wk + n * n + 4 * n + (long long)tp * n;
  const double tiny = 2.220446049250313e-16 * fmax(fabs(lam[0]), fabs(lam[job.nvec - 1])) + 1e-300;
  const double l = lam[tp];
  double dd[SLAR_MAX_N], dl[SLAR_MAX_N], du[SLAR_MAX_N], du2[SLAR_MAX_N], b[SLAR_MAX_N];
  unsigned char ip[SLAR_MAX_N];
  for (int i = 0; i < n; ++i) b[i] = hash_unit((unsigned long long)tp * 1024ull + i);
  for (int it = 0; it < 3; ++it) {
    for (int i = 0; i < n; ++i) {
      dd[i] = d[i] - l;
      dl[i] = i + 1 < n ? e[i] : 0.0;
      du[i] = dl[i];
      du2[i] = 0.0;
    }
    for (int i = 0; i + 1 < n; ++i) {
      if (fabs(dd[i]) >= fabs(dl[i])) {
        if (dd[i] == 0.0) dd[i] = tiny;
        const double f = dl[i] / dd[i];
        dl[i] = f;
        dd[i + 1] -= f * du[i];
        ip[i] = 0;
      } else {
        const double f = dd[i] / dl[i];
        dd[i] = dl[i];
        dl[i] = f;
        const double tmp = du[i];
        du[i] = dd[i + 1];
        dd[i + 1] = tmp - f * dd[i + 1];
        if (i + 2 < n) {
          du2[i] = du[i + 1];
          du[i + 1] = -f * du[i + 1];
        }
        ip[i] = 1;
      }
    }
    if (dd[n - 1] == 0.0) dd[n - 1] = tiny;
    for (int i = 0; i + 1 < n; ++i) {
      if (ip[i]) {
        const double t = b[i] - dl[i] * b[i + 1];
        b[i] = b[i + 1];
        b[i + 1] = t;
      } else {
        b[i + 1] -= dl[i] * b[i];
      }
    }
    b[n - 1] /= dd[n - 1];
    if (n >= 2) b[n - 2] = (b[n - 2] - du[n - 2] * b[n - 1]) / dd[n - 2];
    for (int i = n - 3; i >= 0; --i) b[i] = (b[i] - du[i] * b[i + 1] - du2[i] * b[i + 2]) / dd[i];
    double mx = 0.0;
    for (int i = 0; i < n; ++i) mx = fmax(mx, fabs(b[i]));
    if (!(mx > 0.0) || !isfinite(mx)) {
      for (int i = 0; i < n; ++i) b[i] = hash_unit((unsigned long long)tp * 1024ull + 512ull + i);
      continue;
    }
    double s2 = 0.0;
    for (int i = 0; i < n; ++i) { b[i] /= mx; s2 += b[i] * b[i]; }
    const double inv = 1.0 / sqrt(s2);
    for (int i = 0; i < n; ++i) b[i] *= inv;
  }
  for (int i = 0; i < n; ++i) z[i] = b[i];
}

// CGS2 of the inverse-iteration vectors (largest eigenvalue first), in place in the work
// array
__global__ void __launch_bounds__(256) k_tri_orth(const EigJob* jobs) {
  extern __shared__ double sZ[];            // nvec columns of n
  __shared__ double sc[SLAR_MAX_N];
  __shared__ double red[8];
  const EigJob job = jobs[blockIdx.x];
  if (!tri_active(job)) return;
  const int n = job.n, nv = job.nvec, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* zg = job.work + n * n + 4 * n;
  for (int it = tid; it < nv * n; it += 256) sZ[it] = zg[it];
  __syncthreads();
  for (int t = 0; t < nv; ++t) {
    double* zt = sZ + t * n;
    for (int pass = 0; pass < 2 && t > 0; ++pass) {
      for (int q = warp; q < t; q += 8) {
        double acc = 0.0;
        for (int i = lane; i < n; i += 32) acc += sZ[q * n + i] * zt[i];
        acc = warp_sum_d(acc);
        if (lane == 0) sc[q] = acc;
      }
      __syncthreads();
      for (int i = tid; i < n; i += 256) {
        double acc = 0.0;
        for (int q = 0; q < t; ++q) acc += sc[q] * sZ[q * n + i];
        zt[i] -= acc;
      }
      __syncthreads();
    }
    double ss = 0.0;
    for (int i = tid; i < n; i += 256) ss += zt[i] * zt[i];
    const double nrm2 = block_sum(ss, red);
    const double inv = nrm2 > 0.0 ? 1.0 / sqrt(nrm2) : 0.0;
    for (int i = tid; i < n; i += 256) zt[i] *= inv;
    __syncthreads();
  }
  for (int it = tid; it < nv * n; it += 256) zg[it] = sZ[it];
}

// back-transformation y = H_0 ... H_{n-3} z of TRI_BACK_COLS vectors per CTA, and the
// outputs of EigJob::tri (CTA 0 also writes W and the unused columns of V)
constexpr int TRI_BACK_COLS = 8;

__global__ void __launch_bounds__(256) k_tri_back(const EigJob* jobs) {
  __shared__ double sZ[TRI_BACK_COLS * SLAR_MAX_N];
  __shared__ double sv[SLAR_MAX_N];
  __shared__ double sc[TRI_BACK_COLS];
  const EigJob job = jobs[blockIdx.y];
  if (!tri_active(job)) return;
  const int n = job.n, nv = job.nvec, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int q0 = blockIdx.x * TRI_BACK_COLS;
  const double* wk = job.work;
  const double* tau = wk + n * n;
  const double* lam = wk + n * n + 3 * n;
  if (blockIdx.x == 0 && tid == 0) {
    double kept = 0.0;
    for (int q = 0; q < nv; ++q) {
      const double l = lam[q] > 0.0 ? lam[q] : 0.0;
      job.W[q] = l;
      kept += l;
    }
    for (int q = nv; q < n; ++q) job.W[q] = 0.0;
    if (nv < n) job.W[nv] = fmax(wk[TRI_TRACE] - kept, 0.0);
  }
  if (blockIdx.x == 0)
    for (int it = tid; it < n * (n - nv); it += 256) {
      const int r = it / (n - nv), q = nv + it % (n - nv);
      job.V[r * n + q] = 0.0;
    }
  const int nc = min(TRI_BACK_COLS, nv - q0);
  if (nc <= 0) return;
  for (int it = tid; it < nc * n; it += 256) sZ[it] = wk[n * n + 4 * n + (long long)q0 * n + it];
  __syncthreads();
  for (int k = n - 3; k >= 0; --k) {
    const double t = tau[k];
    if (t == 0.0) continue;
    for (int i = k + 1 + tid; i < n; i += 256) sv[i] = wk[k * n + i];
    __syncthreads();
    if (warp < nc) {
      double acc = 0.0;
      for (int i = k + 1 + lane; i < n; i += 32) acc += sv[i] * sZ[warp * n + i];
      acc = warp_sum_d(acc);
      if (lane == 0) sc[warp] = t * acc;
    }
    __syncthreads();
    const int m = n - k - 1;
    for (int it = tid; it < nc * m; it += 256) {
      const int q = it / m, i = k + 1 + it - q * m;
      sZ[q * n + i] -= sc[q] * sv[i];
    }
    __syncthreads();
  }
  for (int it = tid; it < n * nc; it += 256) {
    const int r = it / nc, q = it % nc;
    job.V[r * n + q0 + q] = sZ[q * n + r];
  }
}

__global__ void k_choose_ranks(RankJob* jobs, int njobs, const double* normF2, double scale) {
  const int j = threadIdx.x;
  if (j >= njobs) return;
  const RankJob jb = jobs[j];
  const double thr = scale * normF2[0];
  double tail = 0.0;
  int k = jb.n;
  // smallest k with sum_{i >= k} max(lam_i, 0) <= thr
  for (int i = jb.n - 1; i >= 0; --i) {
    const double l = jb.W[i] > 0.0 ? jb.W[i] : 0.0;
    if (tail + l <= thr) { tail += l; k = i; } else break;
  }
  if (k < 1) k = 1;
  if (k > jb.cap) {
    k = jb.cap;
    if (jb.capped) atomicOr(jb.capped, 1);
  }
  jb.out[0] = k;
}

__global__ void k_transpose(const double* __restrict__ A, int rows, int cols, double* __restrict__ B) {
  __shared__ double t[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int r = by + y, c = bx + threadIdx.x;
    if (r < rows && c < cols) t[y][threadIdx.x] = A[(long long)r * cols + c];
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int c = bx + y, r = by + threadIdx.x;
    if (r < rows && c < cols) B[(long long)c * rows + r] = t[threadIdx.x][y];
  }
}

__global__ void k_copy_cols(const double* __restrict__ A, int lda, int rows, int cols,
                            double* __restrict__ B, int ldb) {
  const long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= (long long)rows * cols) return;
  const int r = (int)(it / cols), c = (int)(it % cols);
  B[(long long)r * ldb + c] = A[(long long)r * lda + c];
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// several arrays in one launch: element i belongs to segment s with off[s] <= i < off[s + 1]
__global__ void k_to_float_multi(F32Batch bt) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= bt.off[bt.k]) return;
  int s = 0;
  while (i >= bt.off[s + 1]) ++s;
  const long long j = i - bt.off[s];
  bt.b[s][j] = (float)bt.a[s][j];
}

__global__ void k_identity(double* A, int n, int ld) {
  const int it = blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= n * n) return;
  const int i = it / n, j = it % n;
  A[(long long)i * ld + j] = (i == j) ? 1.0 : 0.0;
}

__global__ void k_zero(double* A, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) A[i] = 0.0;
}

}  // namespace

cudaError_t dgemm(int tA, int tB, int M, int N, int K, double alpha, const double* A, int lda,
                  long long sA, const double* B, int ldb, long long sB, double beta, double* C,
                  int ldc, long long sC, int batch, cudaStream_t s) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  const long long tiles32 = (long long)((N + GT - 1) / GT) * ((M + GT - 1) / GT) * batch;
  if (tiles32 >= 148) {
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT, batch);
    slar::count_launch(), k_dgemm<<<grid, 256, 0, s>>>(tA, tB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
  } else if (4 * tiles32 >= 148) {
    dim3 grid((N + 15) / 16, (M + 15) / 16, batch);
    slar::count_launch(), k_dgemm_small<16><<<grid, 256, 0, s>>>(tA, tB, M, N, K, alpha, A, lda, sA, B, ldb, sB,
                                                                beta, C, ldc, sC);
  } else {
    dim3 grid((N + 7) / 8, (M + 7) / 8, batch);
    slar::count_launch(), k_dgemm_small<8><<<grid, 64, 0, s>>>(tA, tB, M, N, K, alpha, A, lda, sA, B, ldb, sB,
                                                              beta, C, ldc, sC);
  }
  return cudaGetLastError();
}

cudaError_t gram_tall(const double* A, long long lda, int m, int n, double* G, double* work,
                      int work_blocks, cudaStream_t s) {
  const int nblk = (m + GR_ROWS - 1) / GR_ROWS;
  if (nblk > work_blocks || n > SLAR_MAX_RANK) return cudaErrorInvalidValue;
  slar::count_launch(), k_gram_partial<<<nblk, 256, 0, s>>>(A, lda, m, n, work);
  const int nn = n * n;
  slar::count_launch(), k_sum_partials<<<(nn + 255) / 256, 256, 0, s>>>(work, nblk, nn, G);
  return cudaGetLastError();
}

static cudaError_t contract_general(const double* X, long long xp, long long xi, long long xc,
                                    const double* Y, long long yp, long long yj, long long yc,
                                    int P, int I, int J, int C, double* out, double* work,
                                    long long work_len, cudaStream_t s) {
  int groups = 1;
  const int tiles = ((I + CT - 1) / CT) * ((J + CT - 1) / CT);
  while (groups * 2 <= P && tiles * groups * 2 <= 296 && (long long)groups * 2 * I * J <= work_len)
    groups *= 2;
  const int pgroup = (P + groups - 1) / groups;
  groups = (P + pgroup - 1) / pgroup;
  dim3 grid((J + CT - 1) / CT, (I + CT - 1) / CT, groups);
  slar::count_launch(), k_contract<<<grid, 256, 0, s>>>(X, xp, xi, xc, Y, yp, yj, yc, P, I, J, C,
                                                       pgroup, work);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nn = I * J;
  slar::count_launch(), k_sum_partials<<<(nn + 255) / 256, 256, 0, s>>>(work, groups, nn, out);
  return cudaGetLastError();
}

cudaError_t contract_last(const double* X, const double* Y, int P, int I, int J, int C,
                          double* out, double* work, long long work_len, cudaStream_t s) {
  return contract_general(X, (long long)I * C, C, 1, Y, (long long)J * C, C, 1, P, I, J, C, out,
                          work, work_len, s);
}

cudaError_t contract_mid(const double* X, const double* Y, int P, int C, int I, int J,
                         double* out, double* work, long long work_len, cudaStream_t s) {
  return contract_general(X, (long long)C * I, 1, I, Y, (long long)C * J, 1, J, P, I, J, C, out,
                          work, work_len, s);
}

// large dynamic shared memory for the Cholesky and Jacobi kernels (called at context creation)
cudaError_t linalg_init_attrs() {
  const int sm_chol = (int)(sizeof(double) * 2 * SLAR_MAX_RANK * (SLAR_MAX_RANK + 1));
  cudaError_t e = cudaFuncSetAttribute(k_chol_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_chol);
  if (e != cudaSuccess) return e;
  size_t sm = sizeof(double) * EIG_SMEM_DOUBLES;
  if (sm < sizeof(double) * SLAR_MAX_N * SLAR_MAX_N) sm = sizeof(double) * SLAR_MAX_N * SLAR_MAX_N;
  e = cudaFuncSetAttribute(k_jacobi<EIG_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_tri_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(double) * SLAR_MAX_N * SLAR_MAX_N));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_tri_orth, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(sizeof(double) * SLAR_MAX_N * SLAR_MAX_RANK));
}

cudaError_t chol_inv(const double* G, int n, double* R, double* Rinv, int* info, cudaStream_t s) {
  if (n > SLAR_MAX_RANK) return cudaErrorInvalidValue;
  const int sm = (int)(sizeof(double) * 2 * SLAR_MAX_RANK * (SLAR_MAX_RANK + 1));
  // one warp for orders up to 32: the factorisation is a chain of n block barriers
  slar::count_launch(), k_chol_inv<<<1, n <= 32 ? 32 : 128, sm, s>>>(G, n, R, Rinv, info);
  return cudaGetLastError();
}

cudaError_t householder_qr(double* A, int m, int n, double* Q, double* R, double* tau,
                           cudaStream_t s) {
  if (n > SLAR_MAX_RANK || m < n) return cudaErrorInvalidValue;
  slar::count_launch(), k_householder<<<1, 256, 0, s>>>(A, m, n, Q, R, tau);
  return cudaGetLastError();
}

cudaError_t eig_batched(const EigJob* jobs_host, int njobs, EigJob* jobs_dev, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  int nmax = 0;
  for (int i = 0; i < njobs; ++i) {
    if (jobs_host[i].n > SLAR_MAX_N || jobs_host[i].n < 1) return cudaErrorInvalidValue;
    nmax = jobs_host[i].n > nmax ? jobs_host[i].n : nmax;
  }
  // compression path: L (n x 64), M and V (64 x 64 each), remaining diagonal; the direct
  // full-rank fallback needs an n x n matrix (n <= 128), which is no larger
  size_t sm = sizeof(double) * EIG_SMEM_DOUBLES;
  if (sm < sizeof(double) * SLAR_MAX_N * SLAR_MAX_N) sm = sizeof(double) * SLAR_MAX_N * SLAR_MAX_N;
  cudaError_t e = cudaMemcpyAsync(jobs_dev, jobs_host, sizeof(EigJob) * njobs,
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  slar::count_launch(), k_jacobi<EIG_THREADS><<<njobs, EIG_THREADS, sm, s>>>(jobs_dev,
                                                                           (long long)(sm / sizeof(double)));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // jobs that k_jacobi handed over (flag in their work array) go through the tridiagonal
  // solver; the kernels return at once for the others
  int ntri = 0, nvmax = 0;
  for (int i = 0; i < njobs; ++i)
    if (jobs_host[i].tri) {
      ++ntri;
      nvmax = jobs_host[i].nvec > nvmax ? jobs_host[i].nvec : nvmax;
    }
  if (ntri == 0) return cudaSuccess;
  slar::count_launch(), k_tri_reduce<<<njobs, TRI_THREADS, sizeof(double) * nmax * nmax, s>>>(jobs_dev);
  const dim3 gb((nvmax + 32 / MS_LANES - 1) / (32 / MS_LANES), njobs);
  slar::count_launch(), k_tri_bisect<<<gb, 32, 0, s>>>(jobs_dev);
  const dim3 gv((nvmax + TRI_EIG_PER_CTA - 1) / TRI_EIG_PER_CTA, njobs);
  slar::count_launch(), k_tri_vec<<<gv, TRI_EIG_PER_CTA, 0, s>>>(jobs_dev);
  slar::count_launch(), k_tri_orth<<<njobs, 256, sizeof(double) * nvmax * nmax, s>>>(jobs_dev);
  const dim3 gt((nvmax + TRI_BACK_COLS - 1) / TRI_BACK_COLS, njobs);
  slar::count_launch(), k_tri_back<<<gt, 256, 0, s>>>(jobs_dev);
  return cudaGetLastError();
}

cudaError_t choose_ranks(const RankJob* jobs_host, int njobs, RankJob* jobs_dev, const double* normF2,
                         double scale, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(jobs_dev, jobs_host, sizeof(RankJob) * njobs,
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  slar::count_launch(), k_choose_ranks<<<1, 32, 0, s>>>(jobs_dev, njobs, normF2, scale);
  return cudaGetLastError();
}

cudaError_t transpose(const double* A, int rows, int cols, double* B, cudaStream_t s) {
  dim3 blk(32, 8), grid((cols + 31) / 32, (rows + 31) / 32);
  slar::count_launch(), k_transpose<<<grid, blk, 0, s>>>(A, rows, cols, B);
  return cudaGetLastError();
}

cudaError_t copy_cols(const double* A, int lda, int rows, int cols, double* B, int ldb,
                      cudaStream_t s) {
  const long long n = (long long)rows * cols;
  if (n == 0) return cudaSuccess;
  slar::count_launch(), k_copy_cols<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(A, lda, rows, cols, B, ldb);
  return cudaGetLastError();
}

cudaError_t to_float(const double* a, float* b, long long n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  slar::count_launch(), k_to_float<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, b, n);
  return cudaGetLastError();
}

void F32Batch::add(const double* src, float* dst, long long n) {
  if (n <= 0) return;
  a[k] = src;
  b[k] = dst;
  off[k + 1] = off[k] + n;
  ++k;
}

cudaError_t to_float_batch(const F32Batch& bt, cudaStream_t s) {
  if (bt.k == 0) return cudaSuccess;
  const long long n = bt.off[bt.k];
  slar::count_launch(), k_to_float_multi<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(bt);
  return cudaGetLastError();
}

cudaError_t fill_identity(double* A, int n, int ld, cudaStream_t s) {
  slar::count_launch(), k_identity<<<(n * n + 255) / 256, 256, 0, s>>>(A, n, ld);
  return cudaGetLastError();
}

cudaError_t fill_zero(double* A, long long n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  slar::count_launch(), k_zero<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(A, n);
  return cudaGetLastError();
}

}  // namespace slar
