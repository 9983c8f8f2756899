// Adaptive-weight LoMaC projection (Sec. 3.2.1-3.2.2; Supp. B), FP64:
//   omega^(mu) = max(|U_v_mu[:,0]|, delta)                         (Supp. B.1)
//   weighted Gram-Schmidt gamma, q1, eta, beta, q2 and the norms     (Supp. B.2)
//   C0, C1_mu, C2 from raw moments (Eq. C0_def, C1_def, C2_def)
//   R(U): raw moments from U (Eq. M from U) then the same coefficients (Supp. B.3)
//   F^{n+1} = F* - R(U(F*)) + R(U^{n+1}) stored as HT(F*) + sum_k dC_k (x) Q_k.
#include "context.cuh"
#include "lomac.cuh"

namespace slar {
namespace {

// One CTA: basis vectors, Gram-Schmidt scalars, Q norms and the flux tables <psi Q_k>.
// Warp m builds the basis of velocity dimension m alone (N_v <= 128 points, lane-strided, sums
// by warp shuffles: no block barrier inside the Gram-Schmidt sequence); the inner product
// <p, q>_{omega^-1} = sum p q wq / omega uses one reciprocal of omega per point.
__global__ void k_lomac_basis(GridDesc g, const double* Uv0, int r0, const double* Uv1, int r1,
                              double delta, double* qv, double* bs, int nmom) {
  extern __shared__ double sh[];
  const int dx = g.dx, dv = g.dv;
  const int Nv = g.N[dx];
  const int tid = threadIdx.x;
  const int m = tid >> 5, lane = tid & 31;
  // sums s[f][m][p] = sum_i vec_f[i] v_i^p dv  (f: omega, q1, q2; p = 0..3)
  double* ssum = sh;                  // [3][2][4]
  double* scal = ssum + 24;           // per m: gamma, eta, beta, n0, n1, n2
  auto warp_sum = [&](double v) -> double {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  };
  if (m < dv) {
    const int mu = dx + m;
    const double* U = m == 0 ? Uv0 : Uv1;
    const int r = m == 0 ? r0 : r1;
    const double wq = g.h[mu];
    double* om = qv + (0 * dv + m) * Nv;
    double* q1 = qv + (1 * dv + m) * Nv;
    double* q2 = qv + (2 * dv + m) * Nv;
    constexpr int PL = SLAR_MAX_N / 32;   // points per lane
    double vv[PL], w[PL], iw[PL], a1[PL], a2[PL];
#pragma unroll
    for (int k = 0; k < PL; ++k) {
      const int i = lane + 32 * k;
      vv[k] = g.lo[mu] + ((double)i + 0.5) * wq;
      w[k] = i < Nv ? fmax(fabs(U[(long long)i * r]), delta) : 0.0;
      iw[k] = i < Nv ? 1.0 / w[k] : 0.0;
      if (i < Nv) om[i] = w[k];
    }
    // <p, q>_{omega^-1} = sum p q wq / omega, with p, q in {omega, v omega, v^2 omega}
    double a = 0.0, b = 0.0, e = 0.0;
#pragma unroll
    for (int k = 0; k < PL; ++k) {
      const double vw = vv[k] * w[k], v2w = vv[k] * vv[k] * w[k];
      a += w[k] * w[k] * wq * iw[k];
      b += vw * w[k] * wq * iw[k];
      e += v2w * w[k] * wq * iw[k];
    }
    const double n0 = warp_sum(a);
    const double gamma = warp_sum(b) / n0;
    const double eta = warp_sum(e) / n0;
    double n1p = 0.0, bp = 0.0;
#pragma unroll
    for (int k = 0; k < PL; ++k) {
      const double vw = vv[k] * w[k], v2w = vv[k] * vv[k] * w[k];
      a1[k] = vw - gamma * w[k];
      n1p += a1[k] * a1[k] * wq * iw[k];
      bp += v2w * a1[k] * wq * iw[k];
    }
    const double n1 = warp_sum(n1p);
    const double beta = warp_sum(bp) / n1;
    double n2p = 0.0;
#pragma unroll
    for (int k = 0; k < PL; ++k) {
      const double v2w = vv[k] * vv[k] * w[k];
      a2[k] = v2w - eta * w[k] - beta * a1[k];
      n2p += a2[k] * a2[k] * wq * iw[k];
      const int i = lane + 32 * k;
      if (i < Nv) {
        q1[i] = a1[k];
        q2[i] = a2[k];
      }
    }
    const double n2 = warp_sum(n2p);
    if (lane == 0) {
      scal[m * 6 + 0] = gamma; scal[m * 6 + 1] = eta; scal[m * 6 + 2] = beta;
      scal[m * 6 + 3] = n0; scal[m * 6 + 4] = n1; scal[m * 6 + 5] = n2;
    }
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      double t[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int k = 0; k < PL; ++k) {
        const double x = f == 0 ? w[k] : (f == 1 ? a1[k] : a2[k]);
        double pw = 1.0;
#pragma unroll
        for (int pp = 0; pp < 4; ++pp) {
          t[pp] += x * pw;
          pw *= vv[k];
        }
      }
#pragma unroll
      for (int pp = 0; pp < 4; ++pp) {
        const double sm = warp_sum(t[pp]) * wq;
        if (lane == 0) ssum[(f * 2 + m) * 4 + pp] = sm;
      }
    }
  }
  __syncthreads();
  // scalars: per m gamma, eta, beta; then nQ0, nQ1[dv], nQ2 (thread 0); the table
  // [nmom][dv+2] one entry per thread, accumulated in registers
  if (tid == 0) {
    double n0p = 1.0;
    for (int m = 0; m < dv; ++m) n0p *= scal[m * 6 + 3];
    for (int m = 0; m < dv; ++m) {
      bs[LS_GAMMA + m] = scal[m * 6 + 0];
      bs[LS_ETA + m] = scal[m * 6 + 1];
      bs[LS_BETA + m] = scal[m * 6 + 2];
    }
    bs[LS_NQ] = n0p;
    double nq2 = 0.0;
    for (int m = 0; m < dv; ++m) {
      double others = 1.0;
      for (int o = 0; o < dv; ++o) if (o != m) others *= scal[o * 6 + 3];
      bs[LS_NQ + 1 + m] = scal[m * 6 + 4] * others;
      nq2 += scal[m * 6 + 5] * others;
    }
    bs[LS_NQ + 1 + dv] = nq2;
  }
  // monomial exponents of the moments (same order as the moment kernels): moment a is the
  // sum of nm[a] monomials v1^p1 v2^p2
  const int nmo = dv == 1 ? 5 : 9;
  const int a = tid / (dv + 2), k = tid - a * (dv + 2);
  if (a >= nmom || a >= nmo) return;
  int ex[2][2] = {{0, 0}, {-1, -1}};
  if (dv == 1) {
    const int p1[5] = {0, 1, 2, 2, 3};
    ex[0][0] = p1[a];
  } else {
    const int t[9][4] = {{0, 0, -1, -1}, {1, 0, -1, -1}, {0, 1, -1, -1}, {2, 0, 0, 2}, {2, 0, -1, -1},
                         {1, 1, -1, -1}, {0, 2, -1, -1}, {3, 0, 1, 2}, {2, 1, 0, 3}};
    ex[0][0] = t[a][0]; ex[0][1] = t[a][1]; ex[1][0] = t[a][2]; ex[1][1] = t[a][3];
  }
  const int nm = ex[1][0] < 0 ? 1 : 2;
  double acc = 0.0;
  for (int mo = 0; mo < nm; ++mo) {
    const int* p = ex[mo];
    if (k == 0) {   // Q0
      double t = 1.0;
      for (int m = 0; m < dv; ++m) t *= ssum[(0 * 2 + m) * 4 + p[m]];
      acc += t;
    } else if (k <= dv) {   // Q1 of dimension k - 1
      const int j = k - 1;
      double t = 1.0;
      for (int m = 0; m < dv; ++m) t *= ssum[((m == j ? 1 : 0) * 2 + m) * 4 + p[m]];
      acc += t;
    } else {   // Q2: sum over the dimensions
      for (int j = 0; j < dv; ++j) {
        double t = 1.0;
        for (int m = 0; m < dv; ++m) t *= ssum[((m == j ? 2 : 0) * 2 + m) * 4 + p[m]];
        acc += t;
      }
    }
  }
  bs[LS_TABLE + a * (dv + 2) + k] = acc;
}

}  // namespace

namespace {

// C from the moments of F* (first dv+2 moment fields)
__global__ void k_coeffs_from_moments(int dv, int NX, const double* bs, const double* mom, double* C) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= NX) return;
  double M1[2], Cl[4];
  for (int m = 0; m < dv; ++m) M1[m] = mom[(long long)(1 + m) * NX + x];
  lomac_coeffs(dv, bs, mom[x], M1, mom[(long long)(1 + dv) * NX + x], Cl);
  for (int k = 0; k < dv + 2; ++k) C[(long long)k * NX + x] = Cl[k];
}

// dC = C~(U) - Cstar, with M2 = 2 (U2 - |E|^2/2) and E the field of U0
__global__ void k_dC_from_U(int dv, int dx, int NX, const double* bs, const double* U, const double* E,
                            const double* Cstar, double* dC) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= NX) return;
  double ep = 0.0;
  for (int m = 0; m < dx; ++m) ep += E[(long long)m * NX + x] * E[(long long)m * NX + x];
  ep *= 0.5;
  double M1[2], Cl[4];
  for (int m = 0; m < dv; ++m) M1[m] = U[(long long)(1 + m) * NX + x];
  lomac_coeffs(dv, bs, U[x], M1, 2.0 * (U[(long long)(1 + dv) * NX + x] - ep), Cl);
  for (int k = 0; k < dv + 2; ++k) dC[(long long)k * NX + x] = Cl[k] - Cstar[(long long)k * NX + x];
}

// U = (M0, M1, M2/2 + |E|^2/2)
__global__ void k_conserved(int dv, int dx, int NX, const double* mom, const double* E, double* U) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= NX) return;
  double ep = 0.0;
  for (int m = 0; m < dx; ++m) ep += E[(long long)m * NX + x] * E[(long long)m * NX + x];
  U[x] = mom[x];
  for (int m = 0; m < dv; ++m) U[(long long)(1 + m) * NX + x] = mom[(long long)(1 + m) * NX + x];
  U[(long long)(1 + dv) * NX + x] = 0.5 * mom[(long long)(1 + dv) * NX + x] + 0.5 * ep;
}

}  // namespace

slar_status conserved_from_moments(slar_ctx* c, const double* mom, const double* E, double* U) {
  slar::count_launch(), k_conserved<<<(c->NX + 255) / 256, 256, 0, c->s>>>(c->dv, c->dx, c->NX, mom, E, U);
  CK(cudaGetLastError());
  return SLAR_OK;
}

slar_status lomac_basis(slar_ctx* c, int slot, double* qv_out, double* bs_out) {
  const HTBuf& h = c->ht[slot];
  const int vl0 = c->dx, vl1 = c->dx + 1;
  slar::count_launch(), k_lomac_basis<<<1, 64, sizeof(double) * 64, c->s>>>(
      c->g, h.U[vl0], h.r[vl0], c->dv == 2 ? h.U[vl1] : nullptr, c->dv == 2 ? h.r[vl1] : 0,
      c->cfg.delta_floor, qv_out, bs_out, c->n_mom);
  CK(cudaGetLastError());
  return SLAR_OK;
}

slar_status coeffs_from_moments(slar_ctx* c, const double* bs, const double* mom, double* C) {
  slar::count_launch(), k_coeffs_from_moments<<<(c->NX + 255) / 256, 256, 0, c->s>>>(c->dv, c->NX, bs, mom, C);
  CK(cudaGetLastError());
  return SLAR_OK;
}

slar_status dC_from_U(slar_ctx* c, const double* bs, const double* U, const double* Cstar, double* dC) {
  // field of U0 (rho = n_i - U0)
  CKS(field_from_M0(c, U, c->E, nullptr, nullptr));
  slar::count_launch(), k_dC_from_U<<<(c->NX + 255) / 256, 256, 0, c->s>>>(c->dv, c->dx, c->NX, bs, U, c->E, Cstar, dC);
  CK(cudaGetLastError());
  return SLAR_OK;
}

// F <- F - R(U(F)) + R(U_target) for the current state (no correction yet).
slar_status lomac_apply(slar_ctx* c, const double* Ut) {
  double* bs = c->lomac_bs;
  double* qv_new = c->lomac_qv;
  CKS(lomac_basis(c, c->cur, qv_new, bs));
  CKS(compute_moments(c, c->cur, false, c->mom, c->dv + 2));
  double* Cstar = c->lomac_C;
  CKS(coeffs_from_moments(c, bs, c->mom, Cstar));
  CKS(dC_from_U(c, bs, Ut, Cstar, c->dC));
  CK(cudaMemcpyAsync(c->qv, qv_new, sizeof(double) * 3 * c->dv * c->g.N[c->dx],
                     cudaMemcpyDeviceToDevice, c->s));
  c->has_corr = 1;
  return SLAR_OK;
}

}  // namespace slar
