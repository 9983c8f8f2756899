// Workspaces and helpers of the macroscopic Newton-Krylov solve shared by macro.cu
// (residual, GMRES, JFNK, time step) and precond.cu (block-circulant preconditioner,
// learned warm start, training-sample recording).
#pragma once

#include "context.cuh"

struct slar_net;

namespace slar {

struct MacroWS {
  int nvec = 0, m = 0;
  double *U = nullptr, *G0 = nullptr, *Ut = nullptr, *Gt = nullptr, *rhs = nullptr;
  double *delta = nullptr, *r = nullptr, *V = nullptr, *Kst[3] = {nullptr, nullptr, nullptr};
  double *mom_star = nullptr, *Ufs = nullptr;
  double *fr = nullptr;        // real staging fields
  double2 *fz = nullptr;       // spectral staging
  double *part = nullptr;      // reduction partials
  double *sc = nullptr;        // device scalars
  double *tot = nullptr;       // totals
  int* gi = nullptr;           // device ints: Arnoldi index j, Krylov count, iterations done
  int nblk = 0;
  cudaGraphExec_t g_pro = nullptr, g_loop = nullptr, g_epi = nullptr;
  cudaGraphExec_t g_loop_pc = nullptr, g_epi_pc = nullptr;   // right-preconditioned variant
  long long n_pro = 0, n_body = 0, n_epi = 0, n_body_pc = 0, n_epi_pc = 0;
  bool graphs = false, graphs_pc = false;

  // block-circulant preconditioner: inverse Fourier-mode blocks P[k][m][m], probe
  // responses, and apply staging
  double2* P = nullptr;        // [NX][m][m]
  double* Rr = nullptr;        // [m][m][NX] responses (real)
  double2* Rz = nullptr;       // [m][m][NX] their spectra
  double* Zr = nullptr;        // [m][NX]
  double2* Zc = nullptr;       // [m][NX]
  // learned warm start
  float* feat = nullptr;       // network input [2m][NX]
  float* ynet = nullptr;       // network output copy [m + m^2][NX]
  double* fstat = nullptr;     // mean, s_U, s_D, probe scales (4m doubles)
  double* vtmp = nullptr;      // [m][NX]
};

constexpr int RED_SEG = 256;
// scalar layout (sc)
constexpr int SC_H = 0;                 // (m+1) x m, m <= 64
constexpr int SC_G = SC_H + 65 * 64;    // m+1
constexpr int SC_CS = SC_G + 65;
constexpr int SC_SN = SC_CS + 64;
constexpr int SC_Y = SC_SN + 64;
constexpr int SC_MISC = SC_Y + 64;      // beta, bnorm, done, jdone, tmp...
enum { M_BETA = 0, M_BNORM, M_DONE, M_JDONE, M_NORM, M_RTOL, M_INF, M_UNORM, M_COEF, M_H, M_INVH,
       M_NI, M_FIRST, M_GRES, M_HC, M_BLK };
constexpr int SC_SIZE = SC_MISC + 16;

inline unsigned nb(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// out = K(U) (mode_g = 0) or G(U) = U - rhs - coef K(U) (mode_g = 1); coef and n_i are
// read from the device scalars (M_COEF, M_NI)
slar_status eval_residual(slar_ctx* c, const double* U, const double* rhs, double* out, int mode_g);
// out[i] (+)= V_i . x for i < nv (V_i = V + i ld), reduced over the vector length nvec
slar_status dot_into(slar_ctx* c, const double* V, long long ld, int nv, const double* x, double* out,
                     int accumulate, const double* done);
slar_status absmax(slar_ctx* c, const double* x, double* out_dev);
__global__ void k_set_scalars(double* misc, double coef, double h, double n_i, double first);
__global__ void k_axpby(const double* a, double s, const double* b, double* out, int n, const double* done);

// preconditioner (precond.cu)
slar_status pc_alloc(slar_ctx* c);
void pc_free(slar_ctx* c);
// probe the Jacobian of G at U (G(U) must be in w->G0) and invert its Fourier-mode blocks
slar_status pc_probe(slar_ctx* c, const double* U);
// out = P B in (B the network block if the device flag M_BLK is set); in may alias out
slar_status pc_apply(slar_ctx* c, const double* in, double* out);
// graph-capturable P B applied to the Arnoldi vector V_j (j read from gi[0]) into w->Zr
slar_status pc_apply_j(slar_ctx* c);
// features of (U^n, U*) into w->feat and the statistics w->fstat
slar_status warm_features(slar_ctx* c, const double* Un, const double* Ustar, float* x_out);
// network inference: w->ynet from w->feat, and the guess U = U* + s_D d
slar_status warm_guess(slar_ctx* c, const double* Ustar, double* U);
__global__ void k_set_misc(double* misc, int slot, double v);
// training sample of the solve just finished (w->U = U^{n+1}, w->Ufs = U*, c->Uc = U^n)
slar_status record_sample(slar_ctx* c);

// network entry points used by the context (net.cu)
cudaError_t net_infer(slar_net* net, const float* x, cudaStream_t s, const float** y);
int net_m(const slar_net* n);
int net_nx(const slar_net* n);
int net_n0(const slar_net* n);
int net_n1(const slar_net* n);
long long net_np(const slar_net* n);

}  // namespace slar
