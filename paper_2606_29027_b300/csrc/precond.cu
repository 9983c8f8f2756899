// Block-circulant right preconditioner of the macroscopic Newton-Krylov solve, the learned
// warm start that sits on top of it, and the recording of training samples (FP64 except the
// network, which is FP32).  An addition to the paper: its JFNK (Sec. 3.2.3) is plain.
//
// Preconditioner.  The Jacobian J of G at the initial guess is probed with one impulse per
// conserved component, r_c = (G(U + h e_c delta_0) - G(U)) / h with h = sqrt(eps)(1 + ||U||).
// For a spatially invariant operator r_c is the c-th block column of a block-circulant
// matrix, whose action on Fourier mode k is the (dv+2) x (dv+2) block
// R(k)[c'][c] = DFT(r_c[c'])(k).  k_invert_blocks inverts every block (Gauss-Jordan with
// partial pivoting in complex FP64; a block whose pivot falls below 1e-14 of its largest
// entry is replaced by the identity) and P y = IDFT(R(k)^{-1} DFT(y)).  With the network
// attached, the Krylov direction is first multiplied point by point by B(x) = I + b(x).
#include <cmath>

#include "context.cuh"
#include "macro.cuh"
#include "spectral.cuh"

namespace slar {
namespace {

constexpr double PIVOT_FLOOR = 1e-14;
constexpr double SCALE_FLOOR = 1e-30;

__global__ void k_impulse(const double* U, double* Ut, int n, int pos, double h) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) Ut[e] = U[e] + (e == pos ? h : 0.0);
}

// response of impulse c: R[(c m + c2) NX + x] = (Gt[c2][x] - G0[c2][x]) / h
__global__ void k_response(const double* Gt, const double* G0, double invh, int c, int m, int NX, double* R) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * NX) return;
  R[(long long)c * m * NX + e] = (Gt[e] - G0[e]) * invh;
}

// P[k][i][j] = (R(k)^{-1})[i][j] with R(k)[i][j] = Rz[(j m + i) NX + k]
__global__ void k_invert_blocks(const double2* __restrict__ Rz, int m, int NX, double2* __restrict__ P) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NX) return;
  double2 A[4][8];
  double scale = 0.0;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      const double2 v = Rz[((long long)j * m + i) * NX + k];
      A[i][j] = v;
      A[i][m + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
      scale = fmax(scale, hypot(v.x, v.y));
    }
  bool ok = scale > 0.0;
  for (int col = 0; col < m && ok; ++col) {
    int piv = col;
    double best = hypot(A[col][col].x, A[col][col].y);
    for (int r = col + 1; r < m; ++r) {
      const double a = hypot(A[r][col].x, A[r][col].y);
      if (a > best) { best = a; piv = r; }
    }
    if (!(best > PIVOT_FLOOR * scale)) { ok = false; break; }
    if (piv != col)
      for (int j = 0; j < 2 * m; ++j) { const double2 t = A[col][j]; A[col][j] = A[piv][j]; A[piv][j] = t; }
    // row col /= pivot
    const double2 p = A[col][col];
    const double den = p.x * p.x + p.y * p.y;
    const double2 ip = make_double2(p.x / den, -p.y / den);
    for (int j = 0; j < 2 * m; ++j) {
      const double2 a = A[col][j];
      A[col][j] = make_double2(a.x * ip.x - a.y * ip.y, a.x * ip.y + a.y * ip.x);
    }
    for (int r = 0; r < m; ++r) {
      if (r == col) continue;
      const double2 f = A[r][col];
      for (int j = 0; j < 2 * m; ++j) {
        const double2 a = A[col][j];
        A[r][j].x -= f.x * a.x - f.y * a.y;
        A[r][j].y -= f.x * a.y + f.y * a.x;
      }
    }
  }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j)
      P[((long long)k * m + i) * m + j] = ok ? A[i][m + j] : make_double2(i == j ? 1.0 : 0.0, 0.0);
}

// Y(k) <- P(k) Y(k), Y [m][NX] complex, in place
__global__ void k_apply_blocks(const double2* __restrict__ P, int m, int NX, double2* __restrict__ Y) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NX) return;
  double2 y[4], z[4];
  for (int j = 0; j < m; ++j) y[j] = Y[(long long)j * NX + k];
  for (int i = 0; i < m; ++i) {
    double2 s = make_double2(0.0, 0.0);
    for (int j = 0; j < m; ++j) {
      const double2 p = P[((long long)k * m + i) * m + j];
      s.x += p.x * y[j].x - p.y * y[j].y;
      s.y += p.x * y[j].y + p.y * y[j].x;
    }
    z[i] = s;
  }
  for (int i = 0; i < m; ++i) Y[(long long)i * NX + k] = z[i];
}

// out[i][x] = v[i][x] + sum_j b[i][j](x) v[j][x] if misc[M_BLK] != 0 (b = network channels
// m + i m + j), else out = v.  v = V + gi[0] n when gi is given (the Arnoldi vector V_j).
__global__ void k_block_apply(const double* __restrict__ V, const int* gi, const float* __restrict__ y,
                              const double* misc, int m, int NX, double* __restrict__ out) {
  if (gi && misc[M_DONE] != 0.0) return;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= NX) return;
  const long long n = (long long)m * NX;
  const double* v = gi ? V + (long long)gi[0] * n : V;
  double a[4];
  for (int j = 0; j < m; ++j) a[j] = v[(long long)j * NX + x];
  const bool blk = misc[M_BLK] != 0.0;
  for (int i = 0; i < m; ++i) {
    double s = a[i];
    if (blk)
      for (int j = 0; j < m; ++j) s += (double)y[(long long)(m + i * m + j) * NX + x] * a[j];
    out[(long long)i * NX + x] = s;
  }
}

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

// feature statistics: CTA c < m: mean and RMS of the fluctuation of Un[c]; CTA m + c: RMS of
// Ustar[c] - Un[c].  st = [mean(m) | s_U(m) | s_D(m)]
__global__ void k_feat_stats(const double* Un, const double* Us, int m, int NX, double* st) {
  __shared__ double red[32];
  const int c = blockIdx.x % m;
  const double* u = Un + (long long)c * NX;
  const double* us = Us + (long long)c * NX;
  if ((int)blockIdx.x < m) {
    double s = 0.0;
    for (int x = threadIdx.x; x < NX; x += blockDim.x) s += u[x];
    const double mean = block_sum(s, red) / NX;
    double q = 0.0;
    for (int x = threadIdx.x; x < NX; x += blockDim.x) { const double d = u[x] - mean; q += d * d; }
    const double rms = sqrt(block_sum(q, red) / NX);
    if (threadIdx.x == 0) { st[c] = mean; st[m + c] = fmax(rms, SCALE_FLOOR); }
  } else {
    double q = 0.0;
    for (int x = threadIdx.x; x < NX; x += blockDim.x) { const double d = us[x] - u[x]; q += d * d; }
    const double rms = sqrt(block_sum(q, red) / NX);
    if (threadIdx.x == 0) st[2 * m + c] = fmax(rms, SCALE_FLOOR);
  }
}

__global__ void k_features(const double* Un, const double* Us, const double* st, int m, int NX, float* x) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NX) return;
  for (int c = 0; c < m; ++c) {
    const double u = Un[(long long)c * NX + p];
    x[(long long)c * NX + p] = (float)((u - st[c]) / st[m + c]);
    x[(long long)(m + c) * NX + p] = (float)((Us[(long long)c * NX + p] - u) / st[2 * m + c]);
  }
}

// U = U* + s_D d
__global__ void k_guess(const double* Us, const double* st, const float* y, int m, int NX, double* U) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NX) return;
  for (int c = 0; c < m; ++c)
    U[(long long)c * NX + p] = Us[(long long)c * NX + p] + st[2 * m + c] * (double)y[(long long)c * NX + p];
}

// t = (U^{n+1} - U*) / s_D
__global__ void k_target(const double* Un1, const double* Us, const double* st, int m, int NX, float* t) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NX) return;
  for (int c = 0; c < m; ++c)
    t[(long long)c * NX + p] =
        (float)((Un1[(long long)c * NX + p] - Us[(long long)c * NX + p]) / st[2 * m + c]);
}

// per-component RMS of G, floored: out[c]
__global__ void k_rms(const double* G, int NX, double* out) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  double q = 0.0;
  for (int x = threadIdx.x; x < NX; x += blockDim.x) { const double g = G[(long long)c * NX + x]; q += g * g; }
  const double r = sqrt(block_sum(q, red) / NX);
  if (threadIdx.x == 0) out[c] = fmax(r, SCALE_FLOOR);
}

// v = -G / rms(G) per component (double and float copies)
__global__ void k_v0(const double* G, const double* sc, int m, int NX, double* v, float* vf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * NX) return;
  const double t = -G[e] / sc[e / NX];
  v[e] = t;
  vf[e] = (float)t;
}

// SplitMix64 (Steele, Lea and Flood 2014): the output for counter value i
__device__ unsigned long long splitmix64(unsigned long long seed, unsigned long long i) {
  unsigned long long z = seed + (i + 1ULL) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// random signs v[e] = +-1 from the top bit of SplitMix64(seed, base + e)
__global__ void k_signs(unsigned long long seed, unsigned long long base, int n, double* v, float* vf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const double t = (splitmix64(seed, base + (unsigned long long)e) >> 63) ? -1.0 : 1.0;
  v[e] = t;
  vf[e] = (float)t;
}

__global__ void k_fd_out(const double* Gt, const double* G0, double invh, int n, float* wf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) wf[e] = (float)((Gt[e] - G0[e]) * invh);
}

// h from the norm of Z: misc[M_H] = misc[M_HC] / ||Z||, misc[M_INVH] = 1 / h
__global__ void k_set_h(const double* part, int nblk, int ldp, double* misc) {
  if (threadIdx.x != 0 || misc[M_DONE] != 0.0) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(long long)b * ldp];
  const double nz = sqrt(fmax(s, 0.0));
  const double h = nz > 0.0 ? misc[M_HC] / nz : misc[M_HC];
  misc[M_H] = h;
  misc[M_INVH] = h != 0.0 ? 1.0 / h : 0.0;
}

__global__ void k_znorm_part(const double* __restrict__ z, int n, double* __restrict__ part, int ldp,
                             const double* misc) {
  if (misc[M_DONE] != 0.0) return;
  __shared__ double red[32];
  double s = 0.0;
  for (int e = blockIdx.x * RED_SEG + threadIdx.x; e < (blockIdx.x + 1) * RED_SEG && e < n; e += blockDim.x)
    s += z[e] * z[e];
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) part[(long long)blockIdx.x * ldp] = t;
}

// spectral part of P on w->Zr (in place)
slar_status spectral_apply(slar_ctx* c) {
  MacroWS* w = c->mw;
  const Spectral& sp = *c->spectral;
  const int m = c->dv + 2;
  CK(sp.forward(w->Zr, w->Zc, m));
  slar::count_launch(), k_apply_blocks<<<nb(c->NX, 128), 128, 0, c->s>>>(w->P, m, c->NX, w->Zc);
  CK(cudaGetLastError());
  CK(sp.inverse(w->Zc, w->Zr, m));
  return SLAR_OK;
}

}  // namespace

__global__ void k_set_misc(double* misc, int slot, double v) {
  if (threadIdx.x == 0) misc[slot] = v;
}

slar_status pc_alloc(slar_ctx* c) {
  MacroWS* w = c->mw;
  const long long NX = c->NX, m = c->dv + 2;
  CK(cudaMalloc(&w->P, sizeof(double2) * NX * m * m));
  CK(cudaMalloc(&w->Rr, sizeof(double) * NX * m * m));
  CK(cudaMalloc(&w->Rz, sizeof(double2) * NX * m * m));
  CK(cudaMalloc(&w->Zr, sizeof(double) * NX * m));
  CK(cudaMalloc(&w->Zc, sizeof(double2) * NX * m));
  CK(cudaMalloc(&w->feat, sizeof(float) * NX * 2 * m));
  CK(cudaMalloc(&w->ynet, sizeof(float) * NX * (m + m * m)));
  CK(cudaMalloc(&w->fstat, sizeof(double) * 4 * m));
  CK(cudaMalloc(&w->vtmp, sizeof(double) * NX * m));
  CK(cudaMemsetAsync(w->ynet, 0, sizeof(float) * NX * (m + m * m), c->s));
  return SLAR_OK;
}

void pc_free(slar_ctx* c) {
  MacroWS* w = c->mw;
  if (!w) return;
  void* ps[] = {w->P, w->Rr, w->Rz, w->Zr, w->Zc, w->feat, w->ynet, w->fstat, w->vtmp};
  for (void* p : ps)
    if (p) cudaFree(p);
}

slar_status pc_probe(slar_ctx* c, const double* U) {
  MacroWS* w = c->mw;
  cudaStream_t s = c->s;
  const int n = w->nvec, NX = c->NX, m = c->dv + 2;
  CKS(dot_into(c, U, 0, 1, U, w->tot + 2, 0, nullptr));
  CK(cudaMemcpyAsync(c->scal_host + 26, w->tot + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double h = std::sqrt(std::ldexp(1.0, -52)) * (1.0 + std::sqrt(c->scal_host[26]));
  for (int comp = 0; comp < m; ++comp) {
    slar::count_launch(), k_impulse<<<nb(n), 256, 0, s>>>(U, w->Ut, n, comp * NX, h);
    CK(cudaGetLastError());
    CKS(eval_residual(c, w->Ut, w->rhs, w->Gt, 1));
    slar::count_launch(), k_response<<<nb(n), 256, 0, s>>>(w->Gt, w->G0, 1.0 / h, comp, m, NX, w->Rr);
    CK(cudaGetLastError());
  }
  CK(c->spectral->forward(w->Rr, w->Rz, m * m));
  slar::count_launch(), k_invert_blocks<<<nb(NX, 128), 128, 0, s>>>(w->Rz, m, NX, w->P);
  CK(cudaGetLastError());
  return SLAR_OK;
}

slar_status pc_apply(slar_ctx* c, const double* in, double* out) {
  MacroWS* w = c->mw;
  const int m = c->dv + 2;
  slar::count_launch(), k_block_apply<<<nb(c->NX), 256, 0, c->s>>>(in, nullptr, w->ynet, w->sc + SC_MISC, m,
                                                                   c->NX, w->Zr);
  CK(cudaGetLastError());
  CKS(spectral_apply(c));
  if (out != w->Zr) CK(cudaMemcpyAsync(out, w->Zr, sizeof(double) * w->nvec, cudaMemcpyDeviceToDevice, c->s));
  return SLAR_OK;
}

slar_status pc_apply_j(slar_ctx* c) {
  MacroWS* w = c->mw;
  const int m = c->dv + 2;
  double* misc = w->sc + SC_MISC;
  slar::count_launch(), k_block_apply<<<nb(c->NX), 256, 0, c->s>>>(w->V, w->gi, w->ynet, misc, m, c->NX, w->Zr);
  CK(cudaGetLastError());
  CKS(spectral_apply(c));
  slar::count_launch(), k_znorm_part<<<w->nblk, 256, 0, c->s>>>(w->Zr, w->nvec, w->part, 72, misc);
  slar::count_launch(), k_set_h<<<1, 32, 0, c->s>>>(w->part, w->nblk, 72, misc);
  CK(cudaGetLastError());
  return SLAR_OK;
}

slar_status warm_features(slar_ctx* c, const double* Un, const double* Ustar, float* x_out) {
  MacroWS* w = c->mw;
  const int m = c->dv + 2;
  slar::count_launch(), k_feat_stats<<<2 * m, 256, 0, c->s>>>(Un, Ustar, m, c->NX, w->fstat);
  slar::count_launch(), k_features<<<nb(c->NX), 256, 0, c->s>>>(Un, Ustar, w->fstat, m, c->NX, x_out);
  CK(cudaGetLastError());
  return SLAR_OK;
}

slar_status warm_guess(slar_ctx* c, const double* Ustar, double* U) {
  MacroWS* w = c->mw;
  const int m = c->dv + 2;
  const float* y = nullptr;
  const long long before = launch_count();
  CK(net_infer(c->net, w->feat, c->s, &y));
  (void)before;
  CK(cudaMemcpyAsync(w->ynet, y, sizeof(float) * (m + m * m) * c->NX, cudaMemcpyDeviceToDevice, c->s));
  slar::count_launch(), k_guess<<<nb(c->NX), 256, 0, c->s>>>(Ustar, w->fstat, w->ynet, m, c->NX, U);
  CK(cudaGetLastError());
  return SLAR_OK;
}

slar_status record_sample(slar_ctx* c) {
  MacroWS* w = c->mw;
  cudaStream_t s = c->s;
  const int m = c->dv + 2, NX = c->NX, n = w->nvec, S = c->rec_S;
  float* dst = c->rec_dst;
  double* misc = w->sc + SC_MISC;
  // x from (U^n, U*), t from U^{n+1} (in w->U)
  CKS(warm_features(c, c->Uc, w->Ufs, dst));
  slar::count_launch(), k_target<<<nb(NX), 256, 0, s>>>(w->U, w->Ufs, w->fstat, m, NX, dst + 2LL * m * NX);
  CK(cudaGetLastError());
  // J and the plain block-circulant P at U*
  slar::count_launch(), k_set_misc<<<1, 1, 0, s>>>(misc, M_BLK, 0.0);
  CKS(eval_residual(c, w->Ufs, w->rhs, w->G0, 1));
  CKS(pc_probe(c, w->Ufs));
  const double hc = std::sqrt(std::ldexp(1.0, -52)) * (1.0 + std::sqrt(c->scal_host[26]));
  float* vf = dst + 3LL * m * NX;
  float* wf = vf + (long long)S * m * NX;
  for (int p = 0; p < S; ++p) {
    if (p == 0) {
      slar::count_launch(), k_rms<<<m, 256, 0, s>>>(w->G0, NX, w->fstat + 3 * m);
      slar::count_launch(), k_v0<<<nb(n), 256, 0, s>>>(w->G0, w->fstat + 3 * m, m, NX, w->vtmp, vf);
    } else {
      const unsigned long long base = ((unsigned long long)c->step * 64ULL + (unsigned long long)p) * (unsigned long long)n;
      slar::count_launch(), k_signs<<<nb(n), 256, 0, s>>>(c->rec_seed, base, n, w->vtmp,
                                                          vf + (long long)p * m * NX);
    }
    CK(cudaGetLastError());
    CKS(pc_apply(c, w->vtmp, w->Zr));
    CKS(dot_into(c, w->Zr, 0, 1, w->Zr, w->tot + 3, 0, nullptr));
    CK(cudaMemcpyAsync(c->scal_host + 27, w->tot + 3, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double nz = std::sqrt(c->scal_host[27]);
    const double h = nz > 0.0 ? hc / nz : hc;
    slar::count_launch(), k_axpby<<<nb(n), 256, 0, s>>>(w->Ufs, h, w->Zr, w->Ut, n, nullptr);
    CKS(eval_residual(c, w->Ut, w->rhs, w->Gt, 1));
    slar::count_launch(), k_fd_out<<<nb(n), 256, 0, s>>>(w->Gt, w->G0, 1.0 / h, n, wf + (long long)p * m * NX);
    CK(cudaGetLastError());
  }
  return SLAR_OK;
}

}  // namespace slar
