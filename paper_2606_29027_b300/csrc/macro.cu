// Implicit macroscopic update closed by the LoMaC-corrected kinetic state and the full time
// step (Sec. 3.2.3, Eq. BE_macro, Eq. BE_nonlinear_system, flowchart; Sec. 4 solver
// settings), FP64:
//   K(U) = -D_x . F(U) + S(U), F from U and the flux moments of F^{n+1}(U) =
//   F* - R(U(F*)) + R(U) (Eq. macro_sys_comp, Eq. electric_field_flux), spectral D_x;
//   G(U) = U - rhs - coef K(U) solved by Jacobian-free Newton-Krylov: GMRES(m) with
//   finite-difference J v, classical Gram-Schmidt applied twice, Givens rotations on
//   device scalars (the host reads one convergence flag per GMRES cycle and one residual
//   norm per Newton step);
//   DIRK3 (Alexander 1977, Thm. 5) for the first two steps (every step with SLAR_DIRK_ONLY),
//   variable-step BDF3 afterwards;
//   SLAR_VP by the third-order commutator-free RK exponential integrator (Eq. slarvp).
#include <algorithm>
#include <cmath>
#include <vector>

#include "context.cuh"
#include "lomac.cuh"
#include "macro.cuh"

namespace slar {

namespace {

// ---------------- reductions ----------------
// part[blk][i] = sum over the block's segment of V_i . w   (i < nv), V_i = V + i*ld
__global__ void k_mdot(const double* __restrict__ V, long long ld, int nv, const double* __restrict__ w,
                       int n, double* __restrict__ part, int ldp, const double* done) {
  if (done && done[0] != 0.0) return;
  const int s0 = blockIdx.x * RED_SEG;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i < nv; i += 8) {
    const double* v = V + i * ld;
    double acc = 0.0;
    for (int e = s0 + lane; e < s0 + RED_SEG && e < n; e += 32) acc += v[e] * w[e];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) part[(long long)blockIdx.x * ldp + i] = acc;
  }
}

// out[i] (+)= sum_blk part[blk][i]
__global__ void k_mdot_fin(const double* part, int nblk, int ldp, int nv, double* out, int accumulate,
                           const double* done) {
  if (done && done[0] != 0.0) return;
  const int i = threadIdx.x;
  if (i >= nv) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(long long)b * ldp + i];
  out[i] = accumulate ? out[i] + s : s;
}

// max that propagates NaN (fmax drops it): a non-finite residual or state must surface as a
// NaN norm so that the Newton loop reports SLAR_ENAN instead of converging on the rest
__device__ __forceinline__ double nan_max(double a, double b) { return (a != a || b != b) ? a + b : fmax(a, b); }

__global__ void k_absmax_part(const double* __restrict__ x, int n, double* part) {
  __shared__ double red[8];
  double m = 0.0;
  for (int e = blockIdx.x * RED_SEG + threadIdx.x; e < (blockIdx.x + 1) * RED_SEG && e < n; e += 256)
    m = nan_max(m, fabs(x[e]));
  for (int o = 16; o > 0; o >>= 1) m = nan_max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t = nan_max(t, red[w]);
    part[blockIdx.x] = t;
  }
}

__global__ void k_absmax_fin(const double* part, int nblk, double* out) {
  if (threadIdx.x != 0) return;
  double t = 0.0;
  for (int b = 0; b < nblk; ++b) t = nan_max(t, part[b]);
  out[0] = t;
}

// out = x / sqrt(*nrm2) ; stores sqrt in *dst
__global__ void k_normalize(const double* x, const double* nrm2, double* out, int n, double* dst,
                            const double* done) {
  if (done && done[0] != 0.0) return;
  const double nr = sqrt(fmax(nrm2[0], 0.0));
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = nr > 0.0 ? x[e] / nr : 0.0;
  if (e == 0 && dst) dst[0] = nr;
}

// ---------------- the residual ----------------
// stage 2 (spectral; stage 1 is the forward transform of U0 and U1): phi, E = -grad phi,
// d_t phi with -Lap(d_t phi) = div(U1), grad(d_t phi)
__global__ void k_spec_fields(Spectral sp, const double2* zin, double2* zout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= sp.NX) return;
  const int dx = sp.dx;
  double k[2];
  if (dx == 1) k[0] = sp.kv[0][i];
  else { k[0] = sp.kv[0][i / sp.n[1]]; k[1] = sp.kv[1][i % sp.n[1]]; }
  double k2 = 0.0;
  for (int m = 0; m < dx; ++m) k2 += k[m] * k[m];
  const double2 rh = make_double2(-zin[i].x, -zin[i].y);   // rho^ = -U0^ for |k| > 0
  double2 ph = make_double2(0.0, 0.0);
  if (k2 > 0.0) ph = make_double2(rh.x / k2, rh.y / k2);
  double2 dv = make_double2(0.0, 0.0);
  for (int m = 0; m < dx; ++m) {
    const double2 z = zin[(long long)(1 + m) * sp.NX + i];
    dv.x += -k[m] * z.y;
    dv.y += k[m] * z.x;
  }
  double2 tp = make_double2(0.0, 0.0);
  if (k2 > 0.0) tp = make_double2(dv.x / k2, dv.y / k2);
  zout[i] = ph;
  for (int m = 0; m < dx; ++m) {
    zout[(long long)(1 + m) * sp.NX + i] = make_double2(k[m] * ph.y, -k[m] * ph.x);        // -i k phi
    zout[(long long)(1 + dx + m) * sp.NX + i] = make_double2(-k[m] * tp.y, k[m] * tp.x);  // i k tp
  }
}

// stage 3: fluxes F[eq][dir] and sources from U, phi, E, grad(d_t phi) and the closure
__global__ void k_flux(int dx, int dv, int NX, int nmom, const double* U, const double* fr2,
                       const double* mom_star, const double* Cstar, const double* bs, double* flux,
                       double* src) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= NX) return;
  const double phi = fr2[x];
  double E[2], gt[2];
  double ep = 0.0;
  for (int m = 0; m < dx; ++m) {
    E[m] = fr2[(long long)(1 + m) * NX + x];
    gt[m] = fr2[(long long)(1 + dx + m) * NX + x];
    ep += E[m] * E[m];
  }
  ep *= 0.5;
  const double U0 = U[x];
  double U1[2];
  for (int m = 0; m < dv; ++m) U1[m] = U[(long long)(1 + m) * NX + x];
  const double U2 = U[(long long)(1 + dv) * NX + x];
  double C[4];
  lomac_coeffs(dv, bs, U0, U1, 2.0 * (U2 - ep), C);
  double dC[4];
  for (int k = 0; k < dv + 2; ++k) dC[k] = C[k] - Cstar[(long long)k * NX + x];
  auto mnew = [&](int a) {
    double s = mom_star[(long long)a * NX + x];
    for (int k = 0; k < dv + 2; ++k) s += bs[LS_TABLE + a * (dv + 2) + k] * dC[k];
    return s;
  };
  const int neq = dv + 2;
  // F[eq][dir] at flux[(eq*dx + dir)*NX + x]
  for (int a = 0; a < dx; ++a) flux[((long long)0 * dx + a) * NX + x] = U1[a];
  if (dv == 1) {
    const double Pi = mnew(3), Q3 = mnew(4);
    flux[((long long)1 * dx + 0) * NX + x] = Pi;
    flux[((long long)2 * dx + 0) * NX + x] = 0.5 * Q3 - phi * gt[0] - U1[0] * phi;
  } else {
    const double P11 = mnew(4), P12 = mnew(5), P22 = mnew(6), Q1 = mnew(7), Q2 = mnew(8);
    flux[((long long)1 * dx + 0) * NX + x] = P11;
    flux[((long long)1 * dx + 1) * NX + x] = P12;
    flux[((long long)2 * dx + 0) * NX + x] = P12;
    flux[((long long)2 * dx + 1) * NX + x] = P22;
    flux[((long long)3 * dx + 0) * NX + x] = 0.5 * Q1 - phi * gt[0] - U1[0] * phi;
    flux[((long long)3 * dx + 1) * NX + x] = 0.5 * Q2 - phi * gt[1] - U1[1] * phi;
  }
  (void)neq;
  (void)nmom;
  for (int b = 0; b < dv; ++b) src[(long long)b * NX + x] = -U0 * E[b];
}

// stage 4: out = K(U) = -div + S   or   out = U - rhs - coef K(U)
__global__ void k_final(int dv, int NX, const double* div, const double* src, const double* U,
                        const double* rhs, const double* coefp, double* out, int mode_g) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= NX) return;
  const double coef = mode_g ? coefp[0] : 0.0;
  for (int e = 0; e < dv + 2; ++e) {
    double K = -div[(long long)e * NX + x];
    if (e >= 1 && e <= dv) K += src[(long long)(e - 1) * NX + x];
    const long long id = (long long)e * NX + x;
    out[id] = mode_g ? (U[id] - rhs[id] - coef * K) : K;
  }
}

__global__ void k_totals(const double* U, int nvar, int NX, double cell, double* out) {
  __shared__ double red[32];
  const int v = blockIdx.x;
  double s = 0.0;
  for (int x = threadIdx.x; x < NX; x += blockDim.x) s += U[(long long)v * NX + x];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[v] = t * cell;
  }
}

__global__ void k_lincomb3(double* out, const double* a, double ca, const double* b, double cb,
                           const double* cc_, double cc, int n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  double s = ca * a[e];
  if (b) s += cb * b[e];
  if (cc_) s += cc * cc_[e];
  out[e] = s;
}

__global__ void k_field_comb(const double* E1, const double* E3, double* Ec, int n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) Ec[e] = -E1[e] / 8.0 + 9.0 * E3[e] / 8.0;
}

}  // namespace

// out = a + s * b (s host scalar)
__global__ void k_axpby(const double* a, double s, const double* b, double* out, int n,
                        const double* done) {
  if (done && done[0] != 0.0) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = a[e] + s * b[e];
}

slar_status macro_alloc(slar_ctx* c) {
  MacroWS* w = new MacroWS();
  c->mw = w;
  w->nvec = (c->dv + 2) * c->NX;
  w->m = c->cfg.krylov_restart;
  w->nblk = (w->nvec + RED_SEG - 1) / RED_SEG;
  const long long n = w->nvec;
  const int nfr = (c->dv + 2) * c->dx + 1 + 2 * c->dx + c->dv + (c->dv + 2) + 4;
  long long total = n * (7 + (w->m + 1) + 3) + (long long)c->n_mom * c->NX + n +
                    (long long)nfr * c->NX + 2LL * ((c->dv + 2) * c->dx + 1 + 2 * c->dx) * c->NX +
                    (long long)w->nblk * 72 + SC_SIZE + 16 + LS_SIZE + 3LL * c->dv * c->g.N[c->dx] +
                    (long long)(c->dv + 2) * c->NX + 64;
  if (cudaMalloc(&c->macro_ws, sizeof(double) * total) != cudaSuccess) return SLAR_ENOMEM;
  if (cudaMalloc(&w->gi, sizeof(int) * 8) != cudaSuccess) return SLAR_ENOMEM;
  c->macro_ws_len = total;
  double* p = c->macro_ws;
  auto take = [&](long long k) { double* q = p; p += k; return q; };
  w->U = take(n); w->G0 = take(n); w->Ut = take(n); w->Gt = take(n); w->rhs = take(n);
  w->delta = take(n); w->r = take(n);
  w->V = take(n * (w->m + 1));
  for (int i = 0; i < 3; ++i) w->Kst[i] = take(n);
  w->mom_star = take((long long)c->n_mom * c->NX);
  w->Ufs = take(n);
  w->fr = take((long long)nfr * c->NX);
  w->fz = reinterpret_cast<double2*>(take(2LL * ((c->dv + 2) * c->dx + 1 + 2 * c->dx) * c->NX));
  w->part = take((long long)w->nblk * 72);
  w->sc = take(SC_SIZE);
  w->tot = take(16);
  c->lomac_bs = take(LS_SIZE);
  c->lomac_qv = take(3LL * c->dv * c->g.N[c->dx]);
  c->lomac_C = take((long long)(c->dv + 2) * c->NX);
  return pc_alloc(c);
}

void macro_free(slar_ctx* c) {
  if (c->mw) {
    if (c->mw->g_pro) cudaGraphExecDestroy(c->mw->g_pro);
    if (c->mw->g_loop) cudaGraphExecDestroy(c->mw->g_loop);
    if (c->mw->g_epi) cudaGraphExecDestroy(c->mw->g_epi);
    if (c->mw->g_loop_pc) cudaGraphExecDestroy(c->mw->g_loop_pc);
    if (c->mw->g_epi_pc) cudaGraphExecDestroy(c->mw->g_epi_pc);
    if (c->mw->gi) cudaFree(c->mw->gi);
    pc_free(c);
  }
  delete c->mw;
  c->mw = nullptr;
}

// out = K(U) (mode_g = 0) or G(U) = U - rhs - coef K(U) (mode_g = 1)
slar_status eval_residual(slar_ctx* c, const double* U, const double* rhs, double* out, int mode_g) {
  MacroWS* w = c->mw;
  const Spectral& sp = *c->spectral;
  const int NX = c->NX, dx = c->dx, dv = c->dv;
  cudaStream_t s = c->s;
  double* fr = w->fr;
  double2* fz = w->fz;
  const int nf1 = 1 + dx;                  // rho, U1
  const int nf2 = 1 + 2 * dx;              // phi, E, grad d_t phi
  const int nflux = (dv + 2) * dx;
  double* fr2 = fr + (long long)nf1 * NX;
  double* flux = fr2 + (long long)nf2 * NX;
  double* src = flux + (long long)nflux * NX;
  double* div = src + (long long)dv * NX;
  double2* z1 = fz;
  double2* z2 = fz + (long long)nflux * NX;
  double* misc = w->sc + SC_MISC;
  // spectra of U0 and U1: rho = n_i - U0 differs from -U0 only in the k = 0 mode, which the
  // Poisson solve sets to zero, so k_spec_fields takes rho^ = -U0^
  CK(sp.forward(U, z1, nf1));
  slar::count_launch(), k_spec_fields<<<nb(NX), 256, 0, s>>>(sp, z1, z2);
  CK(cudaGetLastError());
  CK(sp.inverse(z2, fr2, nf2));
  slar::count_launch(), k_flux<<<nb(NX), 256, 0, s>>>(dx, dv, NX, c->n_mom, U, fr2, w->mom_star, c->lomac_C, c->lomac_bs,
                                flux, src);
  CK(cudaGetLastError());
  CK(sp.div_lines(flux, dv + 2, div));
  slar::count_launch(), k_final<<<nb(NX), 256, 0, s>>>(dv, NX, div, src, U, rhs, misc + M_COEF, out,
                                                       mode_g);
  CK(cudaGetLastError());
  return SLAR_OK;
}

slar_status dot_into(slar_ctx* c, const double* V, long long ld, int nv, const double* x, double* out,
                     int accumulate, const double* done) {
  MacroWS* w = c->mw;
  slar::count_launch(), k_mdot<<<w->nblk, 256, 0, c->s>>>(V, ld, nv, x, w->nvec, w->part, 72, done);
  CK(cudaGetLastError());
  slar::count_launch(), k_mdot_fin<<<1, 128, 0, c->s>>>(w->part, w->nblk, 72, nv, out, accumulate, done);
  CK(cudaGetLastError());
  return SLAR_OK;
}

slar_status absmax(slar_ctx* c, const double* x, double* out_dev) {
  MacroWS* w = c->mw;
  slar::count_launch(), k_absmax_part<<<w->nblk, 256, 0, c->s>>>(x, w->nvec, w->part);
  CK(cudaGetLastError());
  slar::count_launch(), k_absmax_fin<<<1, 32, 0, c->s>>>(w->part, w->nblk, out_dev);
  CK(cudaGetLastError());
  return SLAR_OK;
}

__global__ void k_set_scalars(double* misc, double coef, double h, double n_i, double first) {
  if (threadIdx.x != 0) return;
  misc[M_COEF] = coef;
  misc[M_H] = h;
  misc[M_INVH] = h != 0.0 ? 1.0 / h : 0.0;
  misc[M_NI] = n_i;
  misc[M_FIRST] = first;
  misc[M_HC] = h;
}

namespace {

// ---------------- GMRES as CUDA graphs ----------------
// One Arnoldi iteration reads its index j from device memory, so the same captured body
// serves every iteration; a WHILE conditional node repeats it until the Givens update sets
// the convergence flag or j reaches the restart length (always terminates).

__global__ void k_axpby_j(const double* U, const double* misc, const double* V, const int* gi,
                          double* Ut, int n) {
  if (misc[M_DONE] != 0.0) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) Ut[e] = U[e] + misc[M_H] * V[(long long)gi[0] * n + e];
}

// Ut = U + h Z with h from the device scalars (preconditioned Arnoldi direction Z = P B V_j)
__global__ void k_axpby_h(const double* U, const double* misc, const double* Z, double* Ut, int n) {
  if (misc[M_DONE] != 0.0) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) Ut[e] = U[e] + misc[M_H] * Z[e];
}

// out = sum_{i < k} y_i V_i with k = gi[2] (the GMRES correction before preconditioning)
__global__ void k_comb_y(double* out, int n, const double* V, const double* sc, const int* gi) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int k = gi[2];
  double s = 0.0;
  for (int i = 0; i < k; ++i) s += sc[SC_Y + i] * V[(long long)i * n + e];
  out[e] = s;
}

__global__ void k_diff_j(const double* Gt, const double* G0, const double* misc, const int* gi,
                         double* V, int n) {
  if (misc[M_DONE] != 0.0) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) V[(long long)(gi[0] + 1) * n + e] = (Gt[e] - G0[e]) * misc[M_INVH];
}

// partial dots of w = V_{j+1} with V_0..V_j (which = 0) or with itself (which = 1)
__global__ void k_mdot_j(const double* __restrict__ V, int n, const int* gi, int which,
                         double* __restrict__ part, int ldp, const double* misc) {
  if (misc[M_DONE] != 0.0) return;
  const int j = gi[0];
  const double* w = V + (long long)(j + 1) * n;
  const int nv = which ? 1 : j + 1;
  const int s0 = blockIdx.x * RED_SEG;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i < nv; i += 8) {
    const double* v = which ? w : V + (long long)i * n;
    double acc = 0.0;
    for (int e = s0 + lane; e < s0 + RED_SEG && e < n; e += 32) acc += v[e] * w[e];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) part[(long long)blockIdx.x * ldp + i] = acc;
  }
}

// H[i][j] (+)= sum_blk part[blk][i], hcol[i] = that sum; which = 1: H[j+1][j] = sqrt(sum)
__global__ void k_fin_j(const double* part, int nblk, int ldp, double* sc, int m, const int* gi,
                        int pass, int which) {
  double* misc = sc + SC_MISC;
  if (misc[M_DONE] != 0.0) return;
  const int j = gi[0];
  const int i = threadIdx.x;
  const int nv = which ? 1 : j + 1;
  if (i >= nv) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(long long)b * ldp + i];
  double* H = sc + SC_H;
  if (which) {
    H[(j + 1) * m + j] = sqrt(fmax(s, 0.0));
  } else {
    sc[SC_Y + i] = s;
    H[i * m + j] = pass ? H[i * m + j] + s : s;
  }
}

__global__ void k_orth_j(double* V, int n, const double* sc, const int* gi) {
  if (sc[SC_MISC + M_DONE] != 0.0) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int j = gi[0];
  double s = 0.0;
  for (int i = 0; i <= j; ++i) s += sc[SC_Y + i] * V[(long long)i * n + e];
  V[(long long)(j + 1) * n + e] -= s;
}

__global__ void k_scale_j(double* V, int n, const double* sc, int m, const int* gi) {
  if (sc[SC_MISC + M_DONE] != 0.0) return;
  const int j = gi[0];
  const double nr = sc[SC_H + (j + 1) * m + j];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) V[(long long)(j + 1) * n + e] = nr > 0.0 ? V[(long long)(j + 1) * n + e] / nr : 0.0;
}

// Givens update of column j, residual estimate, convergence flag, j += 1, loop condition
__global__ void k_givens_j(double* sc, int m, int* gi, cudaGraphConditionalHandle loop, int use_cond) {
  if (threadIdx.x != 0) return;
  double* misc = sc + SC_MISC;
  int cont = 0;
  if (misc[M_DONE] == 0.0) {
    const int j = gi[0];
    double* H = sc + SC_H;
    double* g = sc + SC_G;
    double* cs = sc + SC_CS;
    double* sn = sc + SC_SN;
    for (int i = 0; i < j; ++i) {
      const double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
      H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
      H[i * m + j] = t;
    }
    const double a = H[j * m + j], b = H[(j + 1) * m + j];
    const double den = hypot(a, b);
    cs[j] = den > 0.0 ? a / den : 1.0;
    sn[j] = den > 0.0 ? b / den : 0.0;
    H[j * m + j] = den;
    H[(j + 1) * m + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    misc[M_JDONE] = j + 1;
    gi[1] += 1;
    gi[0] = j + 1;
    if (fabs(g[j + 1]) <= misc[M_RTOL] * misc[M_BNORM] || b == 0.0 || j + 1 >= m) misc[M_DONE] = 1.0;
    cont = misc[M_DONE] == 0.0 ? 1 : 0;
  }
  if (use_cond) cudaGraphSetConditional(loop, cont);
}

__global__ void k_gmres_start_g(double* sc, int* gi) {
  if (threadIdx.x != 0) return;
  double* misc = sc + SC_MISC;
  const double beta = sqrt(fmax(misc[M_NORM], 0.0));
  misc[M_BETA] = beta;
  if (misc[M_FIRST] != 0.0) misc[M_BNORM] = beta;
  misc[M_JDONE] = 0;
  for (int i = 0; i < 65; ++i) sc[SC_G + i] = 0.0;
  sc[SC_G] = beta;
  misc[M_DONE] = (beta <= misc[M_RTOL] * misc[M_BNORM] || beta == 0.0) ? 1.0 : 0.0;
  gi[0] = 0;
}

__global__ void k_solve_upper_g(double* sc, int m, int* gi) {
  if (threadIdx.x != 0) return;
  double* H = sc + SC_H;
  double* g = sc + SC_G;
  double* y = sc + SC_Y;
  const int k = (int)sc[SC_MISC + M_JDONE];
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int l = i + 1; l < k; ++l) s -= H[i * m + l] * y[l];
    y[i] = H[i * m + i] != 0.0 ? s / H[i * m + i] : 0.0;
  }
  gi[2] = k;
  sc[SC_MISC + M_GRES] = fabs(g[k]);
}

__global__ void k_update_delta(double* delta, int n, const double* V, const double* sc, const int* gi) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int k = gi[2];
  double s = 0.0;
  for (int i = 0; i < k; ++i) s += sc[SC_Y + i] * V[(long long)i * n + e];
  delta[e] += s;
}

__global__ void k_rtol(double* misc, double rtol) {
  if (threadIdx.x == 0) misc[M_RTOL] = rtol;
}

struct SolveStats {
  int newton = 0, krylov = 0, g_evals = 0;
  double residual = 0.0;
  bool converged = false;
};

// GMRES launch sequences (captured into graphs, or launched directly when profiling)
slar_status gmres_pro(slar_ctx* c) {
  MacroWS* w = c->mw;
  cudaStream_t s = c->s;
  double* misc = w->sc + SC_MISC;
  CKS(dot_into(c, w->r, 0, 1, w->r, misc + M_NORM, 0, nullptr));
  slar::count_launch(), k_gmres_start_g<<<1, 32, 0, s>>>(w->sc, w->gi);
  slar::count_launch(), k_normalize<<<nb(w->nvec), 256, 0, s>>>(w->r, misc + M_NORM, w->V, w->nvec, nullptr,
                                                               misc + M_DONE);
  CK(cudaGetLastError());
  return SLAR_OK;
}

slar_status gmres_body(slar_ctx* c, cudaGraphConditionalHandle h, int use_cond, bool pc) {
  MacroWS* w = c->mw;
  cudaStream_t s = c->s;
  const int n = w->nvec, m = w->m;
  double* sc = w->sc;
  double* misc = sc + SC_MISC;
  if (pc) {
    // right preconditioning: the Jacobian acts on Z = P B V_j, with the finite-difference
    // step h = sqrt(eps) (1 + ||U||) / ||Z|| set on the device by pc_apply_j
    CKS(pc_apply_j(c));
    slar::count_launch(), k_axpby_h<<<nb(n), 256, 0, s>>>(w->U, misc, w->Zr, w->Ut, n);
  } else {
    slar::count_launch(), k_axpby_j<<<nb(n), 256, 0, s>>>(w->U, misc, w->V, w->gi, w->Ut, n);
  }
  CKS(eval_residual(c, w->Ut, w->rhs, w->Gt, 1));
  slar::count_launch(), k_diff_j<<<nb(n), 256, 0, s>>>(w->Gt, w->G0, misc, w->gi, w->V, n);
  for (int pass = 0; pass < 2; ++pass) {
    slar::count_launch(), k_mdot_j<<<w->nblk, 256, 0, s>>>(w->V, n, w->gi, 0, w->part, 72, misc);
    slar::count_launch(), k_fin_j<<<1, 128, 0, s>>>(w->part, w->nblk, 72, sc, m, w->gi, pass, 0);
    slar::count_launch(), k_orth_j<<<nb(n), 256, 0, s>>>(w->V, n, sc, w->gi);
  }
  slar::count_launch(), k_mdot_j<<<w->nblk, 256, 0, s>>>(w->V, n, w->gi, 1, w->part, 72, misc);
  slar::count_launch(), k_fin_j<<<1, 128, 0, s>>>(w->part, w->nblk, 72, sc, m, w->gi, 0, 1);
  slar::count_launch(), k_scale_j<<<nb(n), 256, 0, s>>>(w->V, n, sc, m, w->gi);
  slar::count_launch(), k_givens_j<<<1, 32, 0, s>>>(sc, m, w->gi, h, use_cond);
  CK(cudaGetLastError());
  return SLAR_OK;
}

slar_status gmres_epi(slar_ctx* c, bool pc) {
  MacroWS* w = c->mw;
  cudaStream_t s = c->s;
  slar::count_launch(), k_solve_upper_g<<<1, 32, 0, s>>>(w->sc, w->m, w->gi);
  if (pc) {
    // delta += P B (V y)
    slar::count_launch(), k_comb_y<<<nb(w->nvec), 256, 0, s>>>(w->Zr, w->nvec, w->V, w->sc, w->gi);
    CK(cudaGetLastError());
    CKS(pc_apply(c, w->Zr, w->Zr));
    slar::count_launch(), k_axpby<<<nb(w->nvec), 256, 0, s>>>(w->delta, 1.0, w->Zr, w->delta, w->nvec, nullptr);
  } else {
    slar::count_launch(), k_update_delta<<<nb(w->nvec), 256, 0, s>>>(w->delta, w->nvec, w->V, w->sc, w->gi);
  }
  CK(cudaGetLastError());
  return SLAR_OK;
}

// WHILE-loop graph around one Arnoldi iteration (plain or right-preconditioned)
slar_status capture_loop(slar_ctx* c, bool pc, cudaGraphExec_t* exec) {
  cudaStream_t s = c->s;
  cudaGraph_t gl;
  CK(cudaGraphCreate(&gl, 0));
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, gl, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cn;
  CK(cudaGraphAddNode(&cn, gl, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  CKS(gmres_body(c, h, 1, pc));
  cudaGraph_t body_out;
  CK(cudaStreamEndCapture(s, &body_out));
  CK(cudaGraphInstantiate(exec, gl, 0));
  CK(cudaGraphDestroy(gl));
  return SLAR_OK;
}

slar_status capture_linear(slar_ctx* c, int which, bool pc, cudaGraphExec_t* exec) {
  cudaStream_t s = c->s;
  cudaGraph_t g;
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  if (which == 0) CKS(gmres_pro(c));
  else CKS(gmres_epi(c, pc));
  CK(cudaStreamEndCapture(s, &g));
  CK(cudaGraphInstantiate(exec, g, 0));
  CK(cudaGraphDestroy(g));
  return SLAR_OK;
}

// capture the GMRES graphs (prologue, Arnoldi loop, epilogue) once per context and variant
slar_status build_gmres_graphs(slar_ctx* c, bool pc) {
  CaptureScope scope(c);
  MacroWS* w = c->mw;
  if (!w->g_pro) {
    const long long l0 = launch_count();
    CKS(capture_linear(c, 0, false, &w->g_pro));
    w->n_pro = launch_count() - l0;
    add_launches(-w->n_pro);
  }
  const long long l1 = launch_count();
  CKS(capture_loop(c, pc, pc ? &w->g_loop_pc : &w->g_loop));
  const long long l2 = launch_count();
  CKS(capture_linear(c, 1, pc, pc ? &w->g_epi_pc : &w->g_epi));
  const long long l3 = launch_count();
  (pc ? w->n_body_pc : w->n_body) = l2 - l1;
  (pc ? w->n_epi_pc : w->n_epi) = l3 - l2;
  add_launches(-(l3 - l1));   // captured, not executed
  (pc ? w->graphs_pc : w->graphs) = true;
  return SLAR_OK;
}

// JFNK on G(U) = U - rhs - coef K(U); w->U holds the initial guess and the result.
slar_status jfnk(slar_ctx* c, double coef, double tol_abs, SolveStats* st, bool pc) {
  MacroWS* w = c->mw;
  phase(c, PH_NEWTON);
  cudaStream_t s = c->s;
  const int n = w->nvec;
  double* sc = w->sc;
  double* misc = sc + SC_MISC;
  const double sqeps = std::sqrt(std::ldexp(1.0, -52));
  slar::count_launch(), k_rtol<<<1, 32, 0, s>>>(misc, c->cfg.krylov_tol);
  slar::count_launch(), k_set_scalars<<<1, 32, 0, s>>>(misc, coef, 0.0, c->n_i, 1.0);
  CK(cudaGetLastError());
  const bool use_graphs = !(c->cfg.flags & SLAR_PROFILE_EVAL);
  if (use_graphs && !(pc ? w->graphs_pc : w->graphs)) CKS(build_gmres_graphs(c, pc));
  CKS(eval_residual(c, w->U, w->rhs, w->G0, 1));
  st->g_evals += 1;
  for (int it = 0;; ++it) {
    CKS(absmax(c, w->G0, misc + M_INF));
    CKS(dot_into(c, w->U, 0, 1, w->U, misc + M_UNORM, 0, nullptr));
    CK(cudaMemcpyAsync(c->scal_host, misc, sizeof(double) * 16, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double ginf = c->scal_host[M_INF];
    const double unorm = std::sqrt(c->scal_host[M_UNORM]);
    st->residual = ginf;
    if (!(ginf == ginf)) return set_error(c, SLAR_ENAN, "non-finite Newton residual");
    if (ginf <= tol_abs) { st->converged = true; break; }
    if (it >= c->cfg.newton_max) break;
    // GMRES(m) on J delta = -G0 from delta = 0; J v by a forward difference with
    // h = sqrt(eps) (1 + ||U||) / ||v|| and ||v|| = 1 for the Arnoldi vectors
    const double h = sqeps * (1.0 + unorm);
    CK(cudaMemsetAsync(w->delta, 0, sizeof(double) * n, s));
    CK(cudaMemsetAsync(w->gi, 0, sizeof(int) * 4, s));
    bool first = true;
    int kry = 0;
    while (true) {
      if (first) {
        slar::count_launch(), k_lincomb3<<<nb(n), 256, 0, s>>>(w->r, w->G0, -1.0, nullptr, 0.0, nullptr, 0.0, n);
      } else {
        // r = -G0 - J delta with J delta = (G(U + hd delta) - G0) / hd
        CKS(dot_into(c, w->delta, 0, 1, w->delta, misc + M_NORM, 0, nullptr));
        CK(cudaMemcpyAsync(c->scal_host + 20, misc + M_NORM, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const double dn = std::sqrt(c->scal_host[20]);
        const double hd = sqeps * (1.0 + unorm) / (dn > 0.0 ? dn : 1.0);
        slar::count_launch(), k_axpby<<<nb(n), 256, 0, s>>>(w->U, hd, w->delta, w->Ut, n, nullptr);
        CKS(eval_residual(c, w->Ut, w->rhs, w->Gt, 1));
        slar::count_launch(), k_lincomb3<<<nb(n), 256, 0, s>>>(w->r, w->Gt, -1.0 / hd, w->G0, 1.0 / hd - 1.0,
                                                              nullptr, 0.0, n);
        st->g_evals += 1;
      }
      CK(cudaGetLastError());
      slar::count_launch(), k_set_scalars<<<1, 32, 0, s>>>(misc, coef, h, c->n_i, first ? 1.0 : 0.0);
      if (use_graphs) {
        CK(cudaGraphLaunch(w->g_pro, s));
        CK(cudaGraphLaunch(pc ? w->g_loop_pc : w->g_loop, s));
        CK(cudaGraphLaunch(pc ? w->g_epi_pc : w->g_epi, s));
      } else {
        // launched one by one (profiling): stop where the WHILE node would stop
        CKS(gmres_pro(c));
        for (int j = 0; j < w->m; ++j) {
          CK(cudaMemcpyAsync(c->scal_host + 30, misc + M_DONE, sizeof(double), cudaMemcpyDeviceToHost, s));
          CK(cudaStreamSynchronize(s));
          if (c->scal_host[30] != 0.0) break;
          CKS(gmres_body(c, 0, 0, pc));
        }
        CKS(gmres_epi(c, pc));
      }
      CK(cudaMemcpyAsync(c->scal_host, misc, sizeof(double) * 16, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(c->h_ranks + 12, w->gi, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      const int jd = c->h_ranks[14];
      if (use_graphs)
        add_launches(w->n_pro + (pc ? w->n_epi_pc : w->n_epi) +
                     (long long)(pc ? w->n_body_pc : w->n_body) * (jd > 0 ? jd : 1));
      st->g_evals += c->h_ranks[13] - kry;
      kry = c->h_ranks[13];
      const double* ms = c->scal_host;
      const bool conv = ms[M_GRES] <= ms[M_RTOL] * ms[M_BNORM] || jd == 0;
      first = false;
      if (conv || kry >= c->cfg.krylov_max) break;
    }
    st->krylov += kry;
    slar::count_launch(), k_axpby<<<nb(n), 256, 0, s>>>(w->U, 1.0, w->delta, w->U, n, nullptr);
    CK(cudaGetLastError());
    CKS(eval_residual(c, w->U, w->rhs, w->G0, 1));
    st->g_evals += 1;
    st->newton += 1;
  }
  return SLAR_OK;
}

}  // namespace

namespace {

// E of a slot (HT [+ the state's correction]): M0 -> rho = n_i - M0 -> Poisson
slar_status field_of_slot(slar_ctx* c, int slot, bool with_corr, double* E) {
  phase(c, PH_FIELD);
  CKS(compute_moments(c, slot, with_corr, c->mom, 1));
  return field_from_M0(c, c->mom, E, nullptr, nullptr);
}

struct VPInfo {
  long long entries = 0;
  int aca[3] = {0, 0, 0};
};

// F* = SLAR_VP(F^n; dt) by CF3 (Eq. slarvp): Y2 = exp(dt/3 F(Y1)) Y1,
// Y3 = exp(2dt/3 F(Y2)) Y1, F* = exp(dt (-F(Y1)/12 + 3F(Y3)/4)) Y2, the last being a
// frozen-field advection over 2dt/3 with E_c = -E1/8 + 9E3/8.  Returns the slot of F*.
slar_status slar_vp(slar_ctx* c, double dt, int* out_slot, VPInfo* info) {
  const int S = c->cur;
  int fr[3], k = 0;
  for (int i = 0; i < NSLOT; ++i)
    if (i != S) fr[k++] = i;
  const int A = fr[0], B = fr[1];
  long long e[3] = {0, 0, 0};
  CKS(field_of_slot(c, S, true, c->E1));
  CKS(slar_call(c, S, true, dt / 3.0, c->E1, A, &info->aca[0], &e[0]));
  CKS(field_of_slot(c, A, false, c->E2));
  CKS(slar_call(c, S, true, 2.0 * dt / 3.0, c->E2, B, &info->aca[1], &e[1]));
  CKS(field_of_slot(c, B, false, c->E3));
  slar::count_launch(), k_field_comb<<<nb((long long)c->dx * c->NX), 256, 0, c->s>>>(c->E1, c->E3, c->E, c->dx * c->NX);
  CK(cudaGetLastError());
  CKS(slar_call(c, A, false, 2.0 * dt / 3.0, c->E, B, &info->aca[2], &e[2]));
  c->ht[A].valid = false;
  info->entries = e[0] + e[1] + e[2];
  *out_slot = B;
  return SLAR_OK;
}

// closure data of F* in `slot`: LoMaC basis, moments, C(F*), U(F*) (Newton initial guess)
slar_status make_closure(slar_ctx* c, int slot) {
  MacroWS* w = c->mw;
  phase(c, PH_CLOSURE);
  CKS(lomac_basis(c, slot, c->lomac_qv, c->lomac_bs));
  CKS(compute_moments(c, slot, false, w->mom_star, c->n_mom));
  CKS(coeffs_from_moments(c, c->lomac_bs, w->mom_star, c->lomac_C));
  CKS(field_from_M0(c, w->mom_star, c->E, nullptr, nullptr));
  return conserved_from_moments(c, w->mom_star, c->E, w->Ufs);
}

double host_absmax(slar_ctx* c, const double* x, slar_status* st) {
  *st = absmax(c, x, c->mw->tot);
  if (*st != SLAR_OK) return 0.0;
  cudaMemcpyAsync(c->scal_host, c->mw->tot, sizeof(double), cudaMemcpyDeviceToHost, c->s);
  cudaStreamSynchronize(c->s);
  return c->scal_host[0];
}

void dirk3_tableau(double A[3][3], double cst[3]) {
  double g = 0.4358665215;
  for (int i = 0; i < 60; ++i) {
    const double f = g * g * g - 3 * g * g + 1.5 * g - 1.0 / 6.0;
    const double df = 3 * g * g - 6 * g + 1.5;
    g -= f / df;
  }
  const double b1 = -(6 * g * g - 16 * g + 1) / 4.0, b2 = (6 * g * g - 20 * g + 5) / 4.0;
  const double a[3][3] = {{g, 0, 0}, {(1 - g) / 2.0, g, 0}, {b1, b2, g}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) A[i][j] = a[i][j];
  cst[0] = g;
  cst[1] = (1 + g) / 2.0;
  cst[2] = 1.0;
}

// The BDF3 solve from U* = U(F*) (in w->Ufs): plain JFNK (the paper), or with the
// block-circulant preconditioner, optionally warm-started by the attached network; a
// preconditioned solve that fails is repeated by plain JFNK from U*.
slar_status solve_bdf(slar_ctx* c, double coef, double tol_abs, slar_stats* st) {
  MacroWS* w = c->mw;
  cudaStream_t s = c->s;
  const int n = w->nvec;
  double* misc = w->sc + SC_MISC;
  // the preconditioned (and learned) solve is switched off for kPcOffSteps BDF3 steps after
  // one that did not converge and fell back to plain JFNK: where the block-circulant model of
  // the Jacobian does not hold (strongly non-uniform states at large CFL numbers) each step
  // would otherwise pay for a failed solve and the plain one
  const bool pc_on = c->pc_off == 0;
  if (c->pc_off > 0) c->pc_off -= 1;
  const bool learned = (c->cfg.flags & SLAR_LEARNED) && c->net && pc_on;
  const bool pc = pc_on && (learned || (c->cfg.flags & (SLAR_PRECOND | SLAR_LEARNED)));
  CK(cudaMemcpyAsync(w->U, w->Ufs, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  SolveStats ss;
  if (!pc) {
    CKS(jfnk(c, coef, tol_abs, &ss, false));
  } else {
    phase(c, PH_NEWTON);
    slar::count_launch(), k_set_scalars<<<1, 32, 0, s>>>(misc, coef, 0.0, c->n_i, 1.0);
    slar::count_launch(), k_set_misc<<<1, 1, 0, s>>>(misc, M_BLK, learned ? 1.0 : 0.0);
    CK(cudaGetLastError());
    if (learned) {
      // guess U* + s_D d, kept only if its residual is not larger than that of U*
      CKS(warm_features(c, c->Uc, w->Ufs, w->feat));
      CKS(warm_guess(c, w->Ufs, w->Ut));
      CKS(eval_residual(c, w->Ufs, w->rhs, w->G0, 1));
      CKS(absmax(c, w->G0, w->tot));
      CKS(eval_residual(c, w->Ut, w->rhs, w->Gt, 1));
      CKS(absmax(c, w->Gt, w->tot + 1));
      CK(cudaMemcpyAsync(c->scal_host + 24, w->tot, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      st->g_evals += 2;
      if (c->scal_host[25] <= c->scal_host[24]) {
        CK(cudaMemcpyAsync(w->U, w->Ut, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(w->G0, w->Gt, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        st->guess_used = 1;
      }
    } else {
      CKS(eval_residual(c, w->U, w->rhs, w->G0, 1));
      st->g_evals += 1;
    }
    // the blocks of the previous BDF3 step are reused unless they are missing, were probed for
    // another beta dt, are 8 steps old, or the last solve with them needed more than 2 GMRES
    // iterations beyond the solve right after their probe (or failed)
    const bool probe = c->pc_age < 0 || c->pc_stale || c->pc_age >= kPcMaxAge || coef != c->pc_coef;
    if (probe) {
      CKS(pc_probe(c, w->U));
      st->g_evals += c->dv + 2;
      c->pc_age = 0;
      c->pc_coef = coef;
      st->pc_built = 1;
    } else {
      c->pc_age += 1;
    }
    CKS(jfnk(c, coef, tol_abs, &ss, true));
    if (probe) c->pc_krylov_ref = ss.krylov;
    c->pc_stale = !ss.converged || ss.krylov > c->pc_krylov_ref + 2;
    if (!ss.converged) {
      st->fallback = 1;
      c->pc_off = kPcOffSteps;
      st->newton += ss.newton;
      st->krylov += ss.krylov;
      st->g_evals += ss.g_evals;
      ss = SolveStats();
      CK(cudaMemcpyAsync(w->U, w->Ufs, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      CKS(jfnk(c, coef, tol_abs, &ss, false));
    }
  }
  st->newton += ss.newton;
  st->krylov += ss.krylov;
  st->g_evals += ss.g_evals;
  st->residual = ss.residual;
  st->converged = ss.converged ? 1 : 0;
  return SLAR_OK;
}

}  // namespace

// Differentiate the cubic through (t_{n+1}, U^{n+1}) and the three previous states at t_{n+1}
// (Gear's variable-step BDF3): with t_{n+1} = 0 the nodes are 0, -h_n, -h_n - h_{n-1},
// -h_n - h_{n-1} - h_{n-2}; the Lagrange basis derivatives l_j'(0) give
// U^{n+1} - beta h_n K = sum_j a_j U^{n-j}, a_j = -l_{j+1}'(0) / l_0'(0), beta = 1 / (l_0'(0) h_n).
void bdf3_variable(const double h[3], double a[3], double* beta) {
  const double t[4] = {0.0, -h[0], -h[0] - h[1], -h[0] - h[1] - h[2]};
  double dl[4];
  dl[0] = 0.0;
  for (int m = 1; m < 4; ++m) dl[0] += 1.0 / (t[0] - t[m]);
  for (int j = 1; j < 4; ++j) {
    double num = 1.0, den = 1.0;
    for (int m = 0; m < 4; ++m) {
      if (m == j) continue;
      den *= t[j] - t[m];
      if (m != 0) num *= t[0] - t[m];
    }
    dl[j] = num / den;
  }
  for (int j = 0; j < 3; ++j) a[j] = -dl[j + 1] / dl[0];
  *beta = 1.0 / (dl[0] * h[0]);
}

slar_status step_impl(slar_ctx* c, double dt, slar_stats* out) {
  MacroWS* w = c->mw;
  cudaStream_t s = c->s;
  const int n = w->nvec;
  slar_stats st{};
  st.converged = 1;
  int fslot = -1;
  const long long launches0 = launch_count();
  const long long capped0 = c->rank_capped;
  c->prof_n = 0;
  c->prof_flop = 0.0;
  c->ph_n = 0;
  const bool lomac = (c->cfg.flags & SLAR_LOMAC) != 0;
  if (!lomac) {
    VPInfo vi;
    CKS(slar_vp(c, dt, &fslot, &vi));
    st.entries = vi.entries;
    for (int i = 0; i < 3; ++i) st.aca_rank[i] = vi.aca[i];
    st.n_slar = 3;
    c->ht[c->cur].valid = false;
    c->cur = fslot;
    c->has_corr = 0;
    double* t = c->Uh2; c->Uh2 = c->Uh1; c->Uh1 = c->Uc; c->Uc = t;
    CKS(compute_moments(c, c->cur, false, c->mom, c->dv + 2));
    CKS(field_from_M0(c, c->mom, c->E, nullptr, nullptr));
    CKS(conserved_from_moments(c, c->mom, c->E, c->Uc));
  } else {
    slar_status e0;
    const double un_inf = host_absmax(c, c->Uc, &e0);
    CKS(e0);
    if (!(un_inf == un_inf) || std::isinf(un_inf)) return set_error(c, SLAR_ENAN, "non-finite conserved variables U^n");
    const double tol_abs = c->cfg.newton_tol * std::max(1.0, un_inf);
    if (c->step < 2 || (c->cfg.flags & SLAR_DIRK_ONLY)) {
      double A[3][3], cst[3];
      dirk3_tableau(A, cst);
      for (int i = 0; i < 3; ++i) {
        VPInfo vi;
        CKS(slar_vp(c, cst[i] * dt, &fslot, &vi));
        st.entries += vi.entries;
        for (int q = 0; q < 3; ++q) st.aca_rank[3 * i + q] = vi.aca[q];
        CKS(make_closure(c, fslot));
        // rhs = U^n + dt sum_{j<i} a_ij K_j
        CK(cudaMemcpyAsync(w->rhs, c->Uc, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        for (int j = 0; j < i; ++j)
          slar::count_launch(), k_axpby<<<nb(n), 256, 0, s>>>(w->rhs, dt * A[i][j], w->Kst[j], w->rhs, n, nullptr);
        CK(cudaMemcpyAsync(w->U, w->Ufs, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        SolveStats ss;
        CKS(jfnk(c, dt * A[i][i], tol_abs, &ss, false));
        st.g_evals += ss.g_evals;
        st.newton += ss.newton;
        st.krylov += ss.krylov;
        st.residual = std::max(st.residual, ss.residual);
        st.converged &= ss.converged ? 1 : 0;
        CKS(eval_residual(c, w->U, nullptr, w->Kst[i], 0));
        if (i < 2) c->ht[fslot].valid = false;
      }
      st.n_slar = 9;
    } else {
      VPInfo vi;
      CKS(slar_vp(c, dt, &fslot, &vi));
      st.entries = vi.entries;
      for (int i = 0; i < 3; ++i) st.aca_rank[i] = vi.aca[i];
      st.n_slar = 3;
      CKS(make_closure(c, fslot));
      // variable-step BDF3: U - (a0 U^n + a1 U^{n-1} + a2 U^{n-2}) - beta dt K(U) = 0 (equal
      // steps: 18/11, -9/11, 2/11 and 6/11)
      const double hh[3] = {dt, c->dt_hist[0], c->dt_hist[1]};
      double ab[3], beta;
      bdf3_variable(hh, ab, &beta);
      slar::count_launch(), k_lincomb3<<<nb(n), 256, 0, s>>>(w->rhs, c->Uc, ab[0], c->Uh1, ab[1], c->Uh2, ab[2], n);
      CK(cudaGetLastError());
      const double coef = beta * dt;
      CKS(solve_bdf(c, coef, tol_abs, &st));
      if (c->rec_dst) {
        CKS(record_sample(c));
        st.recorded = 1;
        c->rec_dst = nullptr;
      }
    }
    // F^{n+1} = F* - R(U(F*)) + R(U^{n+1}); history shift
    double* t = c->Uh2; c->Uh2 = c->Uh1; c->Uh1 = c->Uc; c->Uc = t;
    CK(cudaMemcpyAsync(c->Uc, w->U, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    c->ht[c->cur].valid = false;
    c->cur = fslot;
    CKS(dC_from_U(c, c->lomac_bs, c->Uc, c->lomac_C, c->dC));
    CK(cudaMemcpyAsync(c->qv, c->lomac_qv, sizeof(double) * 3 * c->dv * c->g.N[c->dx],
                       cudaMemcpyDeviceToDevice, s));
    c->has_corr = 1;
  }
  for (int i = 0; i < 6; ++i) st.ranks[i] = c->ht[c->cur].r[i];
  // diagnostics: electric energy and totals of U^{n+1}
  phase(c, PH_DIAG);
  CKS(field_from_M0(c, c->Uc, c->E, nullptr, c->Wdev));
  double cell = 1.0;
  for (int m = 0; m < c->dx; ++m) cell *= c->g.h[m];
  slar::count_launch(), k_totals<<<c->dv + 2, 256, 0, s>>>(c->Uc, c->dv + 2, c->NX, cell, w->tot);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(c->scal_host, c->Wdev, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(c->scal_host + 1, w->tot, sizeof(double) * (c->dv + 2), cudaMemcpyDeviceToHost, s));
  phase(c, PH_END);
  CK(cudaStreamSynchronize(s));
  for (int i = 0; i + 1 < c->ph_n; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->ph_ev[i], c->ph_ev[i + 1]));
    if (c->ph_tag[i] < 6) st.phase_ms[c->ph_tag[i]] += ms;
  }
  c->ph_n = 0;
  st.field_energy = c->scal_host[0];
  for (int k = 0; k < c->dv + 2; ++k) st.totals[k] = c->scal_host[1 + k];
  st.eval_flop = c->prof_flop;
  st.eval_ms = 0.0;
  for (int i = 0; i < c->prof_n; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]));
    st.eval_ms += ms;
  }
  c->prof_n = 0;
  st.launches = launch_count() - launches0;
  st.eval_tile = c->eval_tile;
  st.rank_capped = (int)(c->rank_capped - capped0);
  c->step += 1;
  c->dt_hist[1] = c->dt_hist[0];
  c->dt_hist[0] = dt;
  if (out) *out = st;
  bool finite = std::isfinite(st.field_energy);
  for (int k = 0; k < c->dv + 2; ++k) finite = finite && std::isfinite(st.totals[k]);
  if (!finite) return set_error(c, SLAR_ENAN, "non-finite field energy or totals after the step");
  if (!st.converged) return set_error(c, SLAR_ENOCONV, "Newton-Krylov did not converge");
  if (st.rank_capped) return set_error(c, SLAR_ERANK, "rank cap reached with eps unmet (result valid)");
  return SLAR_OK;
}

}  // namespace slar
