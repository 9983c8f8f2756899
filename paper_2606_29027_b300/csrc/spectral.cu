// Spectral operators on the periodic spatial grid (Sec. 3.2.3: "spectral differentiation via
// the FFT" for E, the field-energy flux and the auxiliary Poisson problem; Eq. Poisson,
// Eq. Efromphi).  Hand-written radix-2 complex FFT in shared memory (N a power of two,
// N <= 128), one CTA per line; a 2D transform is a row pass and a column pass.
//
// Symbols: d/dx_m -> i k_m with the Nyquist wavenumber of each dimension set to zero;
// the Laplacian is div(grad), -sum k_m^2, and Poisson's equation is inverted on every mode
// with sum k_m^2 > 0 (phi = 0 elsewhere).  These make gradient, divergence and Laplacian
// algebraically compatible.
#include <cmath>
#include <vector>

#include "context.cuh"
#include "spectral.cuh"

namespace slar {
namespace {

// In-place radix-2 FFTs of `nl` lines of length n held in shared memory (line l starts at
// buf + l * ls, element stride es); all threads of the block cooperate.
__device__ void smem_fft_lines(double2* buf, int n, int logn, int nl, int ls, int es,
                               const double2* tw, int inverse) {
  const int tid = threadIdx.x, nt = blockDim.x;
  // bit-reversal permutation (swap pairs once)
  for (int it = tid; it < nl * n; it += nt) {
    const int l = it / n, i = it - l * n;
    const int r = __brev(i) >> (32 - logn);
    if (r > i) {
      double2* a = buf + l * ls + i * es;
      double2* b = buf + l * ls + r * es;
      const double2 t = *a;
      *a = *b;
      *b = t;
    }
  }
  __syncthreads();
  for (int s = 1; s <= logn; ++s) {
    const int m = 1 << s, half = m >> 1;
    for (int it = tid; it < nl * (n / 2); it += nt) {
      const int l = it / (n / 2), b = it - l * (n / 2);
      const int grp = b / half, j = b - grp * half;
      const int i0 = grp * m + j, i1 = i0 + half;
      double2 w = tw[j * (n / m)];
      if (inverse) w.y = -w.y;
      double2* x0 = buf + l * ls + i0 * es;
      double2* x1 = buf + l * ls + i1 * es;
      const double2 u = *x0, v = *x1;
      const double2 t = make_double2(w.x * v.x - w.y * v.y, w.x * v.y + w.y * v.x);
      *x0 = make_double2(u.x + t.x, u.y + t.y);
      *x1 = make_double2(u.x - t.x, u.y - t.y);
    }
    __syncthreads();
  }
}

// LPB lines of length n per CTA: gather (element stride es, line stride ls) into shared
// memory, transform, scatter.  Batch along blockIdx.y with stride bs.  With rin the lines are
// read from a real array of the same layout (imaginary part 0); with rout only the real part,
// times scale, is written, to a real array of the same layout.
__global__ void k_fft_lines(double2* data, const double* __restrict__ rin, double* __restrict__ rout,
                            double scale, int n, int logn, long long es, long long ls, long long bs,
                            int nlines, int lpb, const double2* tw, int inverse) {
  extern __shared__ double2 buf[];
  const int l0 = blockIdx.x * lpb;
  const int nl = min(lpb, nlines - l0);
  const long long boff = blockIdx.y * bs;
  for (int it = threadIdx.x; it < nl * n; it += blockDim.x) {
    const int l = it / n, i = it - l * n;
    const long long off = boff + (l0 + l) * ls + i * es;
    buf[l * n + i] = rin ? make_double2(rin[off], 0.0) : data[off];
  }
  __syncthreads();
  smem_fft_lines(buf, n, logn, nl, n, 1, tw, inverse);
  for (int it = threadIdx.x; it < nl * n; it += blockDim.x) {
    const int l = it / n, i = it - l * n;
    const long long off = boff + (l0 + l) * ls + i * es;
    if (rout) rout[off] = buf[l * n + i].x * scale;
    else data[off] = buf[l * n + i];
  }
}

// Spectral derivative along one dimension of LPB lines per CTA: forward FFT of the line,
// times i k (Nyquist wavenumber 0), inverse FFT, 1/n; the real part is written to out or added
// to it.  Batch (blockIdx.y) over vectors with strides fvs (input) and ovs (output).  Because
// the 2D DFT factorises, d/dx_m of a field needs transforms along x_m only; a divergence
// sum_m d_m F[.][m] is one such pass per dimension.
__global__ void k_deriv_lines(const double* __restrict__ f, double* out, int n, int logn, long long es, long long ls,
                              int nlines, int lpb, const double2* tw, const double* __restrict__ kv, long long fvs,
                              long long ovs, int accumulate) {
  extern __shared__ double2 buf[];
  const int l0 = blockIdx.x * lpb;
  const int nl = min(lpb, nlines - l0);
  const double* fv = f + blockIdx.y * fvs;
  double* ov = out + blockIdx.y * ovs;
  for (int it = threadIdx.x; it < nl * n; it += blockDim.x) {
    const int l = it / n, i = it - l * n;
    buf[l * n + i] = make_double2(fv[(l0 + l) * ls + i * es], 0.0);
  }
  __syncthreads();
  smem_fft_lines(buf, n, logn, nl, n, 1, tw, 0);
  for (int it = threadIdx.x; it < nl * n; it += blockDim.x) {
    const int i = it % n;
    const double k = kv[i];
    const double2 z = buf[it];
    buf[it] = make_double2(-k * z.y, k * z.x);
  }
  __syncthreads();
  smem_fft_lines(buf, n, logn, nl, n, 1, tw, 1);
  const double scale = 1.0 / n;
  for (int it = threadIdx.x; it < nl * n; it += blockDim.x) {
    const int l = it / n, i = it - l * n;
    const long long off = (l0 + l) * ls + i * es;
    const double v = buf[l * n + i].x * scale;
    ov[off] = accumulate ? ov[off] + v : v;
  }
}

}  // namespace

cudaError_t Spectral::div_lines(const double* F, int nvec, double* div) const {
  // F [nvec][dx][NX] -> div [nvec][NX]; x2 lines are contiguous, x1 lines have stride n[1]
  const int lpb = 2;
  for (int m = dx - 1; m >= 0; --m) {
    const int len = n[m];
    const long long es = (dx == 2 && m == 0) ? n[1] : 1;
    const long long ls = (dx == 2 && m == 0) ? 1 : len;
    const int nlines = NX / len;
    const int thr = len * lpb / 2 < 32 ? 32 : (len * lpb / 2 > 128 ? 128 : len * lpb / 2);
    dim3 grid((nlines + lpb - 1) / lpb, nvec);
    slar::count_launch(), k_deriv_lines<<<grid, thr, sizeof(double2) * lpb * len, s>>>(
        F + (long long)m * NX, div, len, logn[m], es, ls, nlines, lpb, twid[m], kv[m], (long long)dx * NX, NX,
        m == dx - 1 ? 0 : 1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t Spectral::init(int dx_, const int* N, const double* L, cudaStream_t s_) {
  dx = dx_;
  s = s_;
  NX = 1;
  for (int m = 0; m < dx; ++m) {
    n[m] = N[m];
    NX *= N[m];
    logn[m] = 0;
    while ((1 << logn[m]) < n[m]) ++logn[m];
    std::vector<double2> tw(n[m] / 2 > 0 ? n[m] / 2 : 1);
    for (int j = 0; j < n[m] / 2; ++j) {
      const double a = -2.0 * M_PI * j / n[m];
      tw[j] = make_double2(std::cos(a), std::sin(a));
    }
    cudaError_t e = cudaMalloc(&twid[m], sizeof(double2) * tw.size());
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(twid[m], tw.data(), sizeof(double2) * tw.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    std::vector<double> k(n[m]);
    for (int j = 0; j < n[m]; ++j) {
      const int f = j <= n[m] / 2 ? j : j - n[m];
      k[j] = 2.0 * M_PI * f / L[m];
    }
    if (n[m] % 2 == 0) k[n[m] / 2] = 0.0;
    e = cudaMalloc(&kv[m], sizeof(double) * n[m]);
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(kv[m], k.data(), sizeof(double) * n[m], cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void Spectral::release() {
  for (int m = 0; m < 2; ++m) {
    if (twid[m]) cudaFree(twid[m]);
    if (kv[m]) cudaFree(kv[m]);
    twid[m] = nullptr;
    kv[m] = nullptr;
  }
}

// passes of a batched 1D / 2D transform; the first may read real input, the last may write
// the scaled real part
static cudaError_t fft_passes(const Spectral& sp, double2* z, const double* rin, double* rout, double scale,
                              int batch, int inverse) {
  // 2 lines per CTA (one thread per butterfly): the FP64 butterflies of a pass spread over
  // 32 x batch CTAs for 64^2 fields (one B300 SM retires about two FP64 FMAs per clock)
  auto pass = [&](int len, int lg, long long es, long long ls, int nlines, const double2* tw, const double* ri,
                  double* ro) {
    const int lpb = 2;
    const int thr = len * lpb / 2 < 32 ? 32 : (len * lpb / 2 > 128 ? 128 : len * lpb / 2);
    dim3 grid((nlines + lpb - 1) / lpb, batch);
    slar::count_launch(), k_fft_lines<<<grid, thr, sizeof(double2) * lpb * len, sp.s>>>(
        z, ri, ro, scale, len, lg, es, ls, sp.NX, nlines, lpb, tw, inverse);
    return cudaGetLastError();
  };
  if (sp.dx == 1) return pass(sp.n[0], sp.logn[0], 1, sp.n[0], 1, sp.twid[0], rin, rout);
  cudaError_t e = pass(sp.n[1], sp.logn[1], 1, sp.n[1], sp.n[0], sp.twid[1], rin, nullptr);   // rows (x2)
  if (e != cudaSuccess) return e;
  return pass(sp.n[0], sp.logn[0], sp.n[1], 1, sp.n[1], sp.twid[0], nullptr, rout);          // columns (x1)
}

cudaError_t Spectral::fft(double2* z, int batch, int inverse) const {
  return fft_passes(*this, z, nullptr, nullptr, 1.0, batch, inverse);
}

cudaError_t Spectral::forward(const double* f, double2* z, int batch) const {
  return fft_passes(*this, z, f, nullptr, 1.0, batch, 0);
}

cudaError_t Spectral::inverse(double2* z, double* f, int batch) const {
  return fft_passes(*this, z, nullptr, f, 1.0 / NX, batch, 1);
}

}  // namespace slar
