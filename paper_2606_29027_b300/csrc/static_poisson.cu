// Allocation-free variant of the spectral Poisson solve, for callers that cannot allocate
// device memory: for example code that runs while a stream is being recorded into a CUDA
// graph in a capture mode that forbids cudaMalloc, or a host framework that owns a
// fixed pre-reserved device pool and does not let libraries allocate behind its back.
//
// All scratch lives in file-scope static __device__ arrays sized for the largest grid this
// entry point accepts (dx <= 2, at most 128 points per dimension): four spectra of 128^2
// complex values (1 MiB), the twiddle tables and the wavenumbers.  Every GPU that loads the
// library holds these arrays until the process exits.  Host code obtains their device
// addresses with cudaGetSymbolAddress once per device (first call on that device).
#include <cstdio>
#include <mutex>

#include "context.cuh"
#include "spectral.cuh"

namespace slar {
namespace {

constexpr int kStaticMaxN = 128;
constexpr int kStaticFields = 4;  // rho^, phi^, E^ (dx components)

static __device__ __align__(256) double2 g_static_spec[kStaticFields * kStaticMaxN * kStaticMaxN];
static __device__ __align__(256) double2 g_static_twid[2][kStaticMaxN / 2];
static __device__ __align__(256) double g_static_k[2][kStaticMaxN];
static __device__ __align__(256) double g_static_W[1];

struct StaticAddrs {
  double2* spec = nullptr;
  double2* twid = nullptr;
  double* k = nullptr;
  double* W = nullptr;
  bool ready = false;
};
constexpr int kMaxDevices = 64;
StaticAddrs g_addrs[kMaxDevices];
std::mutex g_addr_mutex;

// twiddles exp(-2 pi i j / n) and derivative wavenumbers 2 pi m / L (Nyquist set to 0)
__global__ void k_static_tables(int dx, int n0, int n1, double L0, double L1, double2* twid, double* kv) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  for (int m = 0; m < dx; ++m) {
    const int n = m == 0 ? n0 : n1;
    const double L = m == 0 ? L0 : L1;
    if (t < n / 2) {
      double sn, cs;
      sincospi(-2.0 * t / n, &sn, &cs);
      twid[m * (kStaticMaxN / 2) + t] = make_double2(cs, sn);
    }
    if (t < n) {
      const int f = t <= n / 2 ? t : t - n;
      kv[m * kStaticMaxN + t] = (n % 2 == 0 && t == n / 2) ? 0.0 : 2.0 * 3.14159265358979323846 * f / L;
    }
  }
}

__global__ void k_static_energy(const double* E, int dx, int NX, double cell, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < dx * NX; i += blockDim.x) s += E[i] * E[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[0] = 0.5 * t * cell;
  }
}

bool is_pow2(int n) { return n >= 2 && (n & (n - 1)) == 0; }

// device addresses of the static arrays on the current device (set up on first use)
cudaError_t static_addrs(StaticAddrs** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  StaticAddrs& a = g_addrs[dev];
  if (!a.ready) {
    void* p = nullptr;
    if ((e = cudaGetSymbolAddress(&p, g_static_spec)) != cudaSuccess) return e;
    a.spec = static_cast<double2*>(p);
    if ((e = cudaGetSymbolAddress(&p, g_static_twid)) != cudaSuccess) return e;
    a.twid = static_cast<double2*>(p);
    if ((e = cudaGetSymbolAddress(&p, g_static_k)) != cudaSuccess) return e;
    a.k = static_cast<double*>(p);
    if ((e = cudaGetSymbolAddress(&p, g_static_W)) != cudaSuccess) return e;
    a.W = static_cast<double*>(p);
    a.ready = true;
  }
  *out = &a;
  return cudaSuccess;
}

}  // namespace
}  // namespace slar

using namespace slar;

extern "C" slar_status slar_poisson_field_static(int dx, const int* N, const double* L,
                                                 const double* rho_dev, double* E_dev,
                                                 double* phi_dev, double* energy, void* stream) {
  if (dx < 1 || dx > 2 || !N || !L || !rho_dev || !E_dev) return SLAR_EINVAL;
  for (int m = 0; m < dx; ++m) {
    if (!is_pow2(N[m]) || N[m] > kStaticMaxN) {
      fprintf(stderr, "slar_poisson_field_static: N[%d] = %d must be a power of two <= %d\n", m,
              N[m], kStaticMaxN);
      return SLAR_EINVAL;
    }
    if (!(L[m] > 0.0)) return SLAR_EINVAL;
  }
  StaticAddrs* a = nullptr;
  cudaError_t e = static_addrs(&a);
  if (e != cudaSuccess) return SLAR_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Spectral sp;
  sp.dx = dx;
  sp.s = s;
  sp.NX = 1;
  for (int m = 0; m < dx; ++m) {
    sp.n[m] = N[m];
    sp.NX *= N[m];
    int lg = 0;
    while ((1 << lg) < N[m]) ++lg;
    sp.logn[m] = lg;
    sp.twid[m] = a->twid + m * (kStaticMaxN / 2);
    sp.kv[m] = a->k + m * kStaticMaxN;
  }
  const int NX = sp.NX;
  slar::count_launch(), k_static_tables<<<1, kStaticMaxN, 0, s>>>(dx, N[0], dx > 1 ? N[1] : 1, L[0],
                                                                 dx > 1 ? L[1] : 1.0, a->twid, a->k);
  if (cudaGetLastError() != cudaSuccess) return SLAR_ECUDA;
  double2* z = a->spec;  // z[0] = rho^, z[1] = phi^, z[2..] = E^
  if (sp.forward(rho_dev, z, 1) != cudaSuccess) return SLAR_ECUDA;
  if (spec_poisson_grad(sp, z, z + NX, z + 2 * NX, -1.0) != cudaSuccess) return SLAR_ECUDA;
  if (sp.inverse(z + 2 * NX, E_dev, dx) != cudaSuccess) return SLAR_ECUDA;
  if (phi_dev && sp.inverse(z + NX, phi_dev, 1) != cudaSuccess) return SLAR_ECUDA;
  if (energy) {
    double cell = 1.0;
    for (int m = 0; m < dx; ++m) cell *= L[m] / N[m];
    slar::count_launch(), k_static_energy<<<1, 256, 0, s>>>(E_dev, dx, NX, cell, a->W);
    if (cudaGetLastError() != cudaSuccess) return SLAR_ECUDA;
    if (cudaMemcpyAsync(energy, a->W, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return SLAR_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SLAR_ECUDA;
  }
  return SLAR_OK;
}
