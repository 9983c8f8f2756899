// Field quantities of the Vlasov-Poisson system on the spatial grid: spectral Poisson solve
// (Eq. Poisson, Eq. Efromphi), charge density rho = n_i - M0 (Eq. charge_density) and the
// electric energy W = 1/2 sum |E|^2 dx^dx (Sec. 2.2, e_p = |E|^2 / 2).
#include <cmath>

#include "context.cuh"
#include "spectral.cuh"

namespace slar {
namespace {

__device__ __forceinline__ void kvec(const Spectral& sp, int idx, double* k) {
  if (sp.dx == 1) {
    k[0] = sp.kv[0][idx];
  } else {
    k[0] = sp.kv[0][idx / sp.n[1]];
    k[1] = sp.kv[1][idx % sp.n[1]];
  }
}

__global__ void k_poisson_grad(Spectral sp, const double2* s_hat, double2* phi_hat,
                               double2* grad_hat, double sign) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= sp.NX) return;
  double k[2];
  kvec(sp, i, k);
  double k2 = 0.0;
  for (int m = 0; m < sp.dx; ++m) k2 += k[m] * k[m];
  double2 ph = make_double2(0.0, 0.0);
  if (k2 > 0.0) ph = make_double2(s_hat[i].x / k2, s_hat[i].y / k2);
  if (phi_hat) phi_hat[i] = ph;
  if (grad_hat)
    for (int m = 0; m < sp.dx; ++m)  // sign * i k_m phi
      grad_hat[(long long)m * sp.NX + i] = make_double2(-sign * k[m] * ph.y, sign * k[m] * ph.x);
}

__global__ void k_rho(const double* M0, double n_i, double* rho, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rho[i] = n_i - M0[i];
}

__global__ void k_energy(const double* E, int dx, int NX, double cell, double* out) {
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

}  // namespace

cudaError_t spec_poisson_grad(const Spectral& sp, const double2* s_hat, double2* phi_hat,
                              double2* grad_hat, double sign) {
  slar::count_launch(), k_poisson_grad<<<(sp.NX + 255) / 256, 256, 0, sp.s>>>(sp, s_hat, phi_hat, grad_hat, sign);
  return cudaGetLastError();
}

// E (and phi) from a charge density; W (device scalar) if W_dev != nullptr
slar_status poisson_dev(slar_ctx* c, const double* rho, double* E, double* phi, double* W_dev) {
  const Spectral& sp = *c->spectral;
  double2* z = reinterpret_cast<double2*>(c->spec);
  const int NX = c->NX;
  // z[0] = rho_hat, z[1] = phi_hat, z[2..] = E_hat
  CK(sp.forward(rho, z, 1));
  CK(spec_poisson_grad(sp, z, z + NX, z + 2 * NX, -1.0));
  CK(sp.inverse(z + 2 * NX, E, c->dx));
  if (phi) CK(sp.inverse(z + NX, phi, 1));
  if (W_dev) {
    double cell = 1.0;
    for (int m = 0; m < c->dx; ++m) cell *= c->g.h[m];
    slar::count_launch(), k_energy<<<1, 256, 0, c->s>>>(E, c->dx, NX, cell, W_dev);
    CK(cudaGetLastError());
  }
  return SLAR_OK;
}

namespace {
// out[m] = max_x |E_m(x)| (one block; NaN propagates)
__global__ void k_absmax_rows(const double* E, int rows, int NX, double* out) {
  __shared__ double red[32];
  for (int m = 0; m < rows; ++m) {
    double v = 0.0;
    for (int i = threadIdx.x; i < NX; i += blockDim.x) {
      const double a = fabs(E[(long long)m * NX + i]);
      v = (a != a || v != v) ? a + v : fmax(v, a);
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double u = __shfl_down_sync(0xffffffffu, v, o);
      v = (u != u || v != v) ? u + v : fmax(v, u);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = (red[w] != red[w] || t != t) ? red[w] + t : fmax(t, red[w]);
      out[m] = t;
    }
    __syncthreads();
  }
}
}  // namespace

// Adaptive step size (Sec. 3.2.3 adaptive time stepping; the dimension-wise CFL numbers
// lambda_i = a_i dt / Delta_i of Appendix A): a = max |v_m| in x_m and max |E_m| of the
// current state's field in v_m.
slar_status cfl_dt(slar_ctx* c, double cfl, double dt_max, double* dt) {
  CKS(compute_moments(c, c->cur, true, c->mom, 1));
  CKS(field_from_M0(c, c->mom, c->E, nullptr, nullptr));
  slar::count_launch(), k_absmax_rows<<<1, 256, 0, c->s>>>(c->E, c->dx, c->NX, c->Wdev);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(c->scal_host, c->Wdev, sizeof(double) * c->dx, cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  double rate = 0.0;
  for (int m = 0; m < c->dx; ++m) {
    const int mv = c->dx + m;
    const double lo = c->g.lo[mv], h = c->g.h[mv];
    const double v0 = std::fabs(lo + 0.5 * h), v1 = std::fabs(lo + (c->g.N[mv] - 0.5) * h);
    const double vmax = v0 > v1 ? v0 : v1;
    const double emax = c->scal_host[m];
    if (!(emax == emax)) return set_error(c, SLAR_ENAN, "non-finite field");
    rate = std::fmax(rate, std::fmax(vmax / c->g.h[m], emax / h));
  }
  double d = rate == 0.0 ? dt_max : std::fmin(dt_max, cfl / rate);
  if (c->step >= 2 && c->dt_hist[0] > 0.0 && !(c->cfg.flags & SLAR_DIRK_ONLY))
    d = std::fmin(d, kBdf3RatioMax * c->dt_hist[0]);
  *dt = d;
  return SLAR_OK;
}

slar_status field_from_M0(slar_ctx* c, const double* M0, double* E, double* phi, double* W_dev) {
  double* rho = c->rho;
  slar::count_launch(), k_rho<<<(c->NX + 255) / 256, 256, 0, c->s>>>(M0, c->n_i, rho, c->NX);
  CK(cudaGetLastError());
  return poisson_dev(c, rho, E, phi, W_dev);
}

}  // namespace slar
