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

// ---------------------------------------------------------------------------------------
// G = A^T A for a tall column-major A (m x n, n <= 64): each CTA reduces ROWS rows into a
// partial n x n; a second kernel sums the partials in block order.
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

// out[i][j] = sum_p sum_c X[p][i][c] Y[p][j][c]
__global__ void k_contract_last(const double* __restrict__ X, const double* __restrict__ Y, int P,
                                int I, int J, int C, double* __restrict__ out) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= I || j >= J) return;
  double s = 0.0;
  for (int p = 0; p < P; ++p) {
    const double* x = X + ((long long)p * I + i) * C;
    const double* y = Y + ((long long)p * J + j) * C;
    for (int c = 0; c < C; ++c) s += x[c] * y[c];
  }
  out[(long long)i * J + j] = s;
}

// out[i][j] = sum_p sum_c X[p][c][i] Y[p][c][j]
__global__ void k_contract_mid(const double* __restrict__ X, const double* __restrict__ Y, int P,
                               int C, int I, int J, double* __restrict__ out) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= I || j >= J) return;
  double s = 0.0;
  for (int p = 0; p < P; ++p) {
    const double* x = X + (long long)p * C * I + i;
    const double* y = Y + (long long)p * C * J + j;
    for (int c = 0; c < C; ++c) s += x[(long long)c * I] * y[(long long)c * J];
  }
  out[(long long)i * J + j] = s;
}

// ---------------------------------------------------------------------------------------
// Cholesky G = R^T R (R upper) and R^{-1}, one CTA, n <= 64.
// ---------------------------------------------------------------------------------------
__global__ void k_chol_inv(const double* __restrict__ G, int n, double* __restrict__ R,
                           double* __restrict__ Rinv, int* info) {
  // Column-equilibrated: factor D^{-1} G D^{-1} = Rt^T Rt with D = diag(sqrt(G_ii)), then
  // R = Rt D and R^{-1} = D^{-1} Rt^{-1}.  Equilibration makes the factorisation
  // insensitive to the column scaling of the matrix whose Gram G is.
  extern __shared__ double chol_smem[];
  double (*a)[SLAR_MAX_RANK + 1] = reinterpret_cast<double (*)[SLAR_MAX_RANK + 1]>(chol_smem);
  double (*ri)[SLAR_MAX_RANK + 1] =
      reinterpret_cast<double (*)[SLAR_MAX_RANK + 1]>(chol_smem + SLAR_MAX_RANK * (SLAR_MAX_RANK + 1));
  __shared__ double dsc[SLAR_MAX_RANK];
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  for (int i = tid; i < n; i += blockDim.x) {
    const double gii = G[i * n + i];
    dsc[i] = gii > 0.0 ? sqrt(gii) : 1.0;
  }
  __syncthreads();
  for (int it = tid; it < n * n; it += blockDim.x) {
    const int i = it / n, j = it % n;
    a[i][j] = G[it] / (dsc[i] * dsc[j]);
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      const double dkk = a[k][k];
      if (!(dkk > 0.0)) { bad = k + 1; a[k][k] = 1.0; }
      else a[k][k] = sqrt(dkk);
    }
    __syncthreads();
    const double rkk = a[k][k];
    for (int j = k + 1 + tid; j < n; j += blockDim.x) a[k][j] /= rkk;
    __syncthreads();
    for (int it = tid; it < (n - k - 1) * (n - k - 1); it += blockDim.x) {
      const int i = k + 1 + it / (n - k - 1), j = k + 1 + it % (n - k - 1);
      if (j >= i) a[i][j] -= a[k][i] * a[k][j];
    }
    __syncthreads();
  }
  for (int j = tid; j < n; j += blockDim.x) {
    for (int i = 0; i < n; ++i) ri[i][j] = 0.0;
    ri[j][j] = 1.0 / a[j][j];
    for (int i = j - 1; i >= 0; --i) {
      double s = 0.0;
      for (int k2 = i + 1; k2 <= j; ++k2) s += a[i][k2] * ri[k2][j];
      ri[i][j] = -s / a[i][i];
    }
  }
  __syncthreads();
  for (int it = tid; it < n * n; it += blockDim.x) {
    const int i = it / n, j = it % n;
    R[it] = (j >= i) ? a[i][j] * dsc[j] : 0.0;
    Rinv[it] = ri[i][j] / dsc[i];
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

__global__ void __launch_bounds__(EIG_THREADS) k_jacobi(EigJob* jobs) {
  extern __shared__ double sA[];  // ne x ne  (ne = n rounded up to even)
  __shared__ int pp[SLAR_MAX_N / 2], qq[SLAR_MAX_N / 2];
  __shared__ double cc[SLAR_MAX_N / 2], ss[SLAR_MAX_N / 2];
  __shared__ double red[EIG_THREADS / 32][2];
  __shared__ int stop;
  const EigJob job = jobs[blockIdx.x];
  const int n = job.n;
  const int ne = n + (n & 1);
  const int half = ne / 2;
  const int tid = threadIdx.x;
  double* V = job.work;  // ne x ne row-major eigenvector accumulator in global scratch
  for (int it = tid; it < ne * ne; it += EIG_THREADS) {
    const int i = it / ne, j = it % ne;
    sA[it] = (i < n && j < n) ? job.A[i * n + j] : 0.0;
    V[it] = (i == j) ? 1.0 : 0.0;
  }
  if (tid == 0) stop = 0;
  __syncthreads();
  const int m = ne - 1;  // round-robin over m rounds, index ne-1 fixed
  for (int sweep = 0; sweep < 30; ++sweep) {
    // convergence test: off-diagonal vs diagonal
    double off = 0.0, dia = 0.0;
    for (int it = tid; it < ne * ne; it += EIG_THREADS) {
      const int i = it / ne, j = it % ne;
      const double v = sA[it];
      if (i == j) dia += v * v; else off += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_down_sync(0xffffffffu, off, o);
      dia += __shfl_down_sync(0xffffffffu, dia, o);
    }
    if ((tid & 31) == 0) { red[tid >> 5][0] = off; red[tid >> 5][1] = dia; }
    __syncthreads();
    if (tid == 0) {
      double o2 = 0.0, d2 = 0.0;
      for (int w = 0; w < EIG_THREADS / 32; ++w) { o2 += red[w][0]; d2 += red[w][1]; }
      stop = (o2 <= 1e-26 * d2) || (d2 == 0.0);
    }
    __syncthreads();
    if (stop) break;
    for (int rnd = 0; rnd < m; ++rnd) {
      for (int k = tid; k < half; k += EIG_THREADS) {
        int p, q;
        if (k == 0) { p = rnd; q = ne - 1; }
        else { p = (rnd + k) % m; q = (rnd - k + m) % m; }
        if (p > q) { const int t = p; p = q; q = t; }
        const double apq = sA[p * ne + q];
        double c = 1.0, s = 0.0;
        if (apq != 0.0) {
          const double app = sA[p * ne + p], aqq = sA[q * ne + q];
          const double theta = (aqq - app) / (2.0 * apq);
          const double t = fabs(theta) > 1e150
                               ? 0.5 / theta
                               : (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
          c = 1.0 / sqrt(t * t + 1.0);
          s = t * c;
        }
        pp[k] = p; qq[k] = q; cc[k] = c; ss[k] = s;
      }
      __syncthreads();
      // A <- J^T A J as independent 2x2 blocks (pair a rows, pair b columns)
      for (int it = tid; it < half * half; it += EIG_THREADS) {
        const int ia = it / half, ib = it % half;
        const int pa = pp[ia], qa = qq[ia], pb = pp[ib], qb = qq[ib];
        const double ca = cc[ia], sa = ss[ia], cb = cc[ib], sb = ss[ib];
        const double x00 = sA[pa * ne + pb], x01 = sA[pa * ne + qb];
        const double x10 = sA[qa * ne + pb], x11 = sA[qa * ne + qb];
        // J^T X : rows (p, q) -> (c x_p - s x_q, s x_p + c x_q)
        const double y00 = ca * x00 - sa * x10, y01 = ca * x01 - sa * x11;
        const double y10 = sa * x00 + ca * x10, y11 = sa * x01 + ca * x11;
        // (.) J : cols (p, q) -> (c y_p - s y_q, s y_p + c y_q)
        sA[pa * ne + pb] = cb * y00 - sb * y01;
        sA[pa * ne + qb] = sb * y00 + cb * y01;
        sA[qa * ne + pb] = cb * y10 - sb * y11;
        sA[qa * ne + qb] = sb * y10 + cb * y11;
      }
      for (int it = tid; it < ne * half; it += EIG_THREADS) {
        const int row = it / half, ib = it % half;
        const int pb = pp[ib], qb = qq[ib];
        const double cb = cc[ib], sb = ss[ib];
        const double vp = V[row * ne + pb], vq = V[row * ne + qb];
        V[row * ne + pb] = cb * vp - sb * vq;
        V[row * ne + qb] = sb * vp + cb * vq;
      }
      __syncthreads();
    }
  }
  // sort descending (ties by index) and write
  for (int i = tid; i < n; i += EIG_THREADS) {
    const double li = sA[i * ne + i];
    int pos = 0;
    for (int j = 0; j < n; ++j) {
      const double lj = sA[j * ne + j];
      pos += (lj > li) || (lj == li && j < i);
    }
    job.W[pos] = li;
    for (int r = 0; r < n; ++r) job.V[r * n + pos] = V[r * ne + i];
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
  if (k > jb.cap) k = jb.cap;
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
  dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT, batch);
  slar::count_launch(), k_dgemm<<<grid, 256, 0, s>>>(tA, tB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
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

cudaError_t contract_last(const double* X, const double* Y, int P, int I, int J, int C,
                          double* out, cudaStream_t s) {
  dim3 blk(16, 16), grid((J + 15) / 16, (I + 15) / 16);
  slar::count_launch(), k_contract_last<<<grid, blk, 0, s>>>(X, Y, P, I, J, C, out);
  return cudaGetLastError();
}

cudaError_t contract_mid(const double* X, const double* Y, int P, int C, int I, int J,
                         double* out, cudaStream_t s) {
  dim3 blk(16, 16), grid((J + 15) / 16, (I + 15) / 16);
  slar::count_launch(), k_contract_mid<<<grid, blk, 0, s>>>(X, Y, P, C, I, J, out);
  return cudaGetLastError();
}

cudaError_t chol_inv(const double* G, int n, double* R, double* Rinv, int* info, cudaStream_t s) {
  if (n > SLAR_MAX_RANK) return cudaErrorInvalidValue;
  const int sm = (int)(sizeof(double) * 2 * SLAR_MAX_RANK * (SLAR_MAX_RANK + 1));
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_chol_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  slar::count_launch(), k_chol_inv<<<1, 256, sm, s>>>(G, n, R, Rinv, info);
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
  const int ne = nmax + (nmax & 1);
  const size_t sm = sizeof(double) * ne * ne;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(double) * SLAR_MAX_N * SLAR_MAX_N));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  cudaError_t e = cudaMemcpyAsync(jobs_dev, jobs_host, sizeof(EigJob) * njobs,
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  slar::count_launch(), k_jacobi<<<njobs, EIG_THREADS, sm, s>>>(jobs_dev);
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
