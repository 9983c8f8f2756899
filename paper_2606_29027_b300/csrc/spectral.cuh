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
  // div[v] = sum_m d_m F[v][m] (spectral derivatives, one line pass per dimension);
  // F [nvec][dx][NX] real, div [nvec][NX] real
  cudaError_t div_lines(const double* F, int nvec, double* div) const;
};

// spectral-space operators (field.cu).  All spectra are [NX] complex per field.
// phi_hat = s_hat / |k|^2 (0 where |k| = 0); grad_hat[m] = i k_m phi_hat (sign = +1) or
// -i k_m phi_hat (sign = -1, E = -grad phi).
cudaError_t spec_poisson_grad(const Spectral& sp, const double2* s_hat, double2* phi_hat,
                              double2* grad_hat, double sign);

}  // namespace slar
