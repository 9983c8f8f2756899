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

// one 1D complex FFT per CTA over `lines` lines of length n with element stride `es` and
// line stride `ls` (in complex elements), batch along blockIdx.y with stride bs.
__global__ void k_fft_lines(double2* data, int n, int logn, long long es, long long ls, long long bs,
                            const double2* tw, int inverse) {
  extern __shared__ double2 buf[];
  double2* line = data + blockIdx.y * bs + blockIdx.x * ls;
  const int tid = threadIdx.x;
  for (int i = tid; i < n; i += blockDim.x) {
    const int rev = __brev(i) >> (32 - logn);
    buf[rev] = line[i * es];
  }
  __syncthreads();
  for (int s = 1; s <= logn; ++s) {
    const int m = 1 << s, half = m >> 1;
    for (int b = tid; b < n / 2; b += blockDim.x) {
      const int grp = b / half, j = b - grp * half;
      const int i0 = grp * m + j, i1 = i0 + half;
      double2 w = tw[j * (n / m)];          // exp(-2 pi i j / m)
      if (inverse) w.y = -w.y;
      const double2 u = buf[i0], v = buf[i1];
      const double2 t = make_double2(w.x * v.x - w.y * v.y, w.x * v.y + w.y * v.x);
      buf[i0] = make_double2(u.x + t.x, u.y + t.y);
      buf[i1] = make_double2(u.x - t.x, u.y - t.y);
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += blockDim.x) line[i * es] = buf[i];
}

__global__ void k_real_to_cplx(const double* __restrict__ f, double2* __restrict__ z, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = make_double2(f[i], 0.0);
}

__global__ void k_cplx_to_real(const double2* __restrict__ z, double* __restrict__ f, long long n,
                               double scale) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) f[i] = z[i].x * scale;
}

}  // namespace

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

cudaError_t Spectral::fft(double2* z, int batch, int inverse) const {
  if (dx == 1) {
    slar::count_launch(), k_fft_lines<<<dim3(1, batch), n[0] / 2 > 0 ? (n[0] / 2 < 64 ? n[0] / 2 : 64) : 1,
                  sizeof(double2) * n[0], s>>>(z, n[0], logn[0], 1, n[0], NX, twid[0], inverse);
    return cudaGetLastError();
  }
  // rows (along x2, contiguous), then columns (along x1, stride n1)
  const int t1 = n[1] / 2 < 64 ? n[1] / 2 : 64;
  slar::count_launch(), k_fft_lines<<<dim3(n[0], batch), t1 > 0 ? t1 : 1, sizeof(double2) * n[1], s>>>(
      z, n[1], logn[1], 1, n[1], NX, twid[1], inverse);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int t0 = n[0] / 2 < 64 ? n[0] / 2 : 64;
  slar::count_launch(), k_fft_lines<<<dim3(n[1], batch), t0 > 0 ? t0 : 1, sizeof(double2) * n[0], s>>>(
      z, n[0], logn[0], n[1], 1, NX, twid[0], inverse);
  return cudaGetLastError();
}

cudaError_t Spectral::forward(const double* f, double2* z, int batch) const {
  const long long tot = (long long)batch * NX;
  slar::count_launch(), k_real_to_cplx<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(f, z, tot);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return fft(z, batch, 0);
}

cudaError_t Spectral::inverse(double2* z, double* f, int batch) const {
  cudaError_t e = fft(z, batch, 1);
  if (e != cudaSuccess) return e;
  const long long tot = (long long)batch * NX;
  slar::count_launch(), k_cplx_to_real<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(z, f, tot, 1.0 / NX);
  return cudaGetLastError();
}

}  // namespace slar
