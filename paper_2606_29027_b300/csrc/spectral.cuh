// Spectral toolkit on the periodic spatial grid (see spectral.cu).
#pragma once

#include <cuda_runtime.h>

namespace slar {

struct Spectral {
  int dx = 0;
  int n[2] = {1, 1};
  int logn[2] = {0, 0};
  int NX = 1;
  cudaStream_t s = nullptr;
  double2* twid[2] = {nullptr, nullptr};  // exp(-2 pi i j / n), j < n/2
  double* kv[2] = {nullptr, nullptr};     // derivative wavenumbers (Nyquist = 0)

  cudaError_t init(int dx, const int* N, const double* L, cudaStream_t s);
  void release();
  // in-place batched complex FFT of `batch` spatial fields (inverse unscaled)
  cudaError_t fft(double2* z, int batch, int inverse) const;
  // real fields -> spectra / spectra -> real fields (inverse scaled by 1/NX; z is used as
  // scratch and holds no defined values afterwards)
  cudaError_t forward(const double* f, double2* z, int batch) const;
  cudaError_t inverse(double2* z, double* f, int batch) const;
};

// spectral-space operators (field.cu).  All spectra are [NX] complex per field.
// phi_hat = s_hat / |k|^2 (0 where |k| = 0); grad_hat[m] = i k_m phi_hat (sign = +1) or
// -i k_m phi_hat (sign = -1, E = -grad phi).
cudaError_t spec_poisson_grad(const Spectral& sp, const double2* s_hat, double2* phi_hat,
                              double2* grad_hat, double sign);
// div_hat = sum_m i k_m v_hat[m]  for `nvec` vectors of dx components each:
// v_hat layout [vec][m][NX], out [vec][NX]
cudaError_t spec_div(const Spectral& sp, const double2* v_hat, int nvec, double2* out);

}  // namespace slar
