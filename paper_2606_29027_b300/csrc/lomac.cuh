// LoMaC basis scalars layout and the closed-form coefficients (Supp. B.2, Eq. C0_def,
// C1_def, C2_def), shared by the projection and the macroscopic residual.
#pragma once

#include "context.cuh"

namespace slar {

// layout of the device array of basis scalars
enum {
  LS_GAMMA = 0,   // [dv]
  LS_ETA = 2,     // [dv]
  LS_BETA = 4,    // [dv]
  LS_NQ = 6,      // ||Q0||^2, ||Q1_mu||^2 [dv], ||Q2||^2
  LS_TABLE = 12,  // <psi_a Q_k>_v, [n_mom][dv+2]
  LS_SIZE = 12 + 9 * 4
};

// C0, C1_mu, C2 of raw moments M0, M1[dv], M2
__device__ __forceinline__ void lomac_coeffs(int dv, const double* bs, double M0, const double* M1,
                                             double M2, double* C) {
  C[0] = M0 / bs[LS_NQ];
  double eta = 0.0;
  for (int m = 0; m < dv; ++m) eta += bs[LS_ETA + m];
  double num2 = M2 - eta * M0;
  for (int m = 0; m < dv; ++m) {
    const double t = M1[m] - bs[LS_GAMMA + m] * M0;
    C[1 + m] = t / bs[LS_NQ + 1 + m];
    num2 -= bs[LS_BETA + m] * t;
  }
  C[1 + dv] = num2 / bs[LS_NQ + 1 + dv];
}

slar_status lomac_basis(slar_ctx* c, int slot, double* qv_out, double* bs_out);
slar_status coeffs_from_moments(slar_ctx* c, const double* bs, const double* mom, double* C);
slar_status dC_from_U(slar_ctx* c, const double* bs, const double* U, const double* Cstar, double* dC);

}  // namespace slar
