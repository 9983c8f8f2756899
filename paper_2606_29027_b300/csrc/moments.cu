// Velocity moments of an HT state (Sec. 2, Eq. raw moments; flux moments of
// Eq. macro_sys_comp) by contracting the velocity leaves with monomial weights and going
// up the tree, plus the exact moments of the separable LoMaC correction (Supp. B.2).
// Midpoint quadrature in v (Supp. B.1).  FP64.
//
// Moment order: M0, M1_1..M1_dv, M2, <v_a v_b f> (a <= b), <|v|^2 v_a f>.
#include "context.cuh"

namespace slar {
namespace {

constexpr int MAXMON = 2;   // monomials per moment
constexpr int MAXMOM = 9;

struct MomentTable {
  int n;
  int nmon[MAXMOM];
  int e[MAXMOM][MAXMON][2];   // exponents (p1, p2) of v1, v2
};

MomentTable make_table(int dv) {
  MomentTable t{};
  int i = 0;
  auto add = [&](int p1, int p2, int q1 = -1, int q2 = -1) {
    t.nmon[i] = 1;
    t.e[i][0][0] = p1; t.e[i][0][1] = p2;
    if (q1 >= 0) { t.nmon[i] = 2; t.e[i][1][0] = q1; t.e[i][1][1] = q2; }
    ++i;
  };
  if (dv == 1) {
    add(0, 0); add(1, 0); add(2, 0); add(2, 0); add(3, 0);
  } else {
    add(0, 0); add(1, 0); add(0, 1); add(2, 0, 0, 2);
    add(2, 0); add(1, 1); add(0, 2);
    add(3, 0, 1, 2); add(2, 1, 0, 3);
  }
  t.n = i;
  return t;
}

__device__ __forceinline__ double vpow(double v, int p) {
  double r = 1.0;
  for (int i = 0; i < p; ++i) r *= v;
  return r;
}

// lv[m][p][a] = sum_j U_{dx+m}[j][a] v_j^p dv   (p = 0..3)
__global__ void k_leaf_moments(GridDesc g, const double* U0, int r0, const double* U1, int r1,
                               double* lv, int ldr) {
  const int m = blockIdx.y;            // velocity dimension
  const int p = blockIdx.z;            // power
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  const double* U = m == 0 ? U0 : U1;
  const int r = m == 0 ? r0 : r1;
  if (a >= r) return;
  const int mu = g.dx + m;
  const int n = g.N[mu];
  double s = 0.0;
  for (int j = 0; j < n; ++j) {
    const double v = g.lo[mu] + ((double)j + 0.5) * g.h[mu];
    s += U[(long long)j * r + a] * vpow(v, p);
  }
  lv[((long long)m * 4 + p) * ldr + a] = s * g.h[mu];
}

// d = 4, first stage: m34[mom][q] = sum_mon sum_{c,e} B34[q][c][e] lv0[p1][c] lv1[p2][e], one
// CTA per (q, mom), a thread per c (the e-sum in four accumulators), the c-sum by shuffles:
// B300 retires about two FP64 FMAs per clock per SM, so the r34 r2 r3 FMAs of a moment are
// spread over r34 SMs and their dependent chains cut fourfold
__global__ void k_mom_m34(MomentTable tab, const double* B34, int r2, int r3, const double* lv, int ldr,
                          double* m34) {
  __shared__ double red[2];
  const int q = blockIdx.x, mom = blockIdx.y, c = threadIdx.x;   // 64 threads >= r2
  double s = 0.0;
  if (c < r2) {
    const double* B = B34 + ((long long)q * r2 + c) * r3;
    for (int mo = 0; mo < tab.nmon[mom]; ++mo) {
      const double* l0 = lv + (0 * 4 + tab.e[mom][mo][0]) * ldr;
      const double* l1 = lv + (1 * 4 + tab.e[mom][mo][1]) * ldr;
      double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
      int e = 0;
      for (; e + 4 <= r3; e += 4) {
        t0 += B[e] * l1[e];
        t1 += B[e + 1] * l1[e + 1];
        t2 += B[e + 2] * l1[e + 2];
        t3 += B[e + 3] * l1[e + 3];
      }
      for (; e < r3; ++e) t0 += B[e] * l1[e];
      s += l0[c] * ((t0 + t1) + (t2 + t3));
    }
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) m34[mom * 64 + q] = red[0] + red[1];
}

// d = 4, second stage: t12[mom][p] = sum_q Broot[p][q] m34[mom][q]
__global__ void k_mom_t12(const double* Broot, int rl, int r34, const double* m34, double* t12) {
  const int mom = blockIdx.x, p = threadIdx.x;
  if (p >= rl) return;
  const double* b = Broot + p * r34;
  const double* m = m34 + mom * 64;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int q = 0;
  for (; q + 4 <= r34; q += 4) {
    a0 += b[q] * m[q];
    a1 += b[q + 1] * m[q + 1];
    a2 += b[q + 2] * m[q + 2];
    a3 += b[q + 3] * m[q + 3];
  }
  for (; q < r34; ++q) a0 += b[q] * m[q];
  t12[mom * 64 + p] = (a0 + a1) + (a2 + a3);
}

// d = 2: t12[mom][a] = sum_b Broot[a][b] lv0[p1][b] (Broot is r0 x r1, the velocity leaf has
// rank r1)
__global__ void k_mom_root_1d(MomentTable tab, int r1, const double* Broot, int r0, const double* lv, int ldr,
                              double* t12) {
  const int mom = blockIdx.x;
  for (int a = threadIdx.x; a < r0; a += blockDim.x) {
    double s = 0.0;
    for (int mo = 0; mo < tab.nmon[mom]; ++mo) {
      const double* l0 = lv + (0 * 4 + tab.e[mom][mo][0]) * ldr;
      for (int b = 0; b < r1; ++b) s += Broot[a * r1 + b] * l0[b];
    }
    t12[mom * 64 + a] = s;
  }
}

// d = 4: Bt[mom][a][b] = sum_p B12[p][a][b] t12[mom][p]
__global__ void k_mom_bt(const double* B12, int r0, int r1, int r12, const double* t12, double* Bt) {
  const int mom = blockIdx.y;
  const int it = blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= r0 * r1) return;
  double s = 0.0;
  for (int p = 0; p < r12; ++p) s += B12[(long long)p * r0 * r1 + it] * t12[mom * 64 + p];
  Bt[(long long)mom * r0 * r1 + it] = s;
}

// field[mom][i] for d = 2: sum_a U0[i][a] t12[mom][a]
__global__ void k_mom_field_1d(const double* U0, int N0, int r0, const double* t12, double* out,
                               int NX) {
  const int mom = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N0) return;
  double s = 0.0;
  for (int a = 0; a < r0; ++a) s += U0[(long long)i * r0 + a] * t12[mom * 64 + a];
  out[(long long)mom * NX + i] = s;
}

// moments of the separable correction: out[mom][x] += sum_terms dC_k(x) prod_mu sum_j vec v^p dv
__global__ void k_corr_moments(GridDesc g, MomentTable tab, const double* dC, const double* qv,
                               double* out, int nmom) {
  const int mom = blockIdx.y;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (mom >= nmom || x >= g.NX) return;
  const int dx = g.dx, dv = g.dv;
  const int Nv = g.N[dx];
  // velocity sums s[f][m][p] of omega (f=0), q1 (f=1), q2 (f=2)
  double acc = 0.0;
  for (int mo = 0; mo < tab.nmon[mom]; ++mo) {
    double vs[3][2];
    for (int f = 0; f < 3; ++f)
      for (int m = 0; m < dv; ++m) {
        const int mu = dx + m;
        const int p = tab.e[mom][mo][m];
        const double* vec = qv + ((long long)f * dv + m) * Nv;
        double s = 0.0;
        for (int j = 0; j < Nv; ++j) {
          const double v = g.lo[mu] + ((double)j + 0.5) * g.h[mu];
          s += vec[j] * vpow(v, p);
        }
        vs[f][m] = s * g.h[mu];
      }
    // term order: Q0, Q1_j, Q2 pieces (as in the evaluator)
    double t = dC[x];
    for (int m = 0; m < dv; ++m) t *= vs[0][m];
    acc += t;
    for (int j = 0; j < dv; ++j) {
      t = dC[(long long)(1 + j) * g.NX + x];
      for (int m = 0; m < dv; ++m) t *= (m == j ? vs[1][m] : vs[0][m]);
      acc += t;
    }
    for (int j = 0; j < dv; ++j) {
      t = dC[(long long)(1 + dv) * g.NX + x];
      for (int m = 0; m < dv; ++m) t *= (m == j ? vs[2][m] : vs[0][m]);
      acc += t;
    }
  }
  out[(long long)mom * g.NX + x] += acc;
}

}  // namespace

slar_status compute_moments(slar_ctx* c, int slot, bool with_corr, double* out, int nmom) {
  cudaStream_t s = c->s;
  const HTBuf& h = c->ht[slot];
  if (!h.valid) return set_error(c, SLAR_EINVAL, "no HT state");
  const MomentTable tab = make_table(c->dv);
  if (nmom > tab.n) nmom = tab.n;
  const GridDesc& g = c->g;
  const int ldr = 64;
  double* lv = c->lvec;              // [2][4][64]
  double* t12 = lv + 2 * 4 * 64;     // [9][64]
  double* Bt = t12 + MAXMOM * 64;    // [9][64*64]
  double* m34 = Bt + MAXMOM * 64 * 64;   // [9][64]
  const int dx = c->dx;
  const int vl0 = dx, vl1 = dx + 1;
  dim3 g1((64 + 63) / 64, c->dv, 4);
  slar::count_launch(), k_leaf_moments<<<g1, 64, 0, s>>>(g, h.U[vl0], h.r[vl0], c->dv == 2 ? h.U[vl1] : nullptr,
                                  c->dv == 2 ? h.r[vl1] : 0, lv, ldr);
  CK(cudaGetLastError());
  if (c->d == 4) {
    slar::count_launch(), k_mom_m34<<<dim3(h.r[5], nmom), 64, 0, s>>>(tab, h.B34, h.r[2], h.r[3], lv, ldr, m34);
    CK(cudaGetLastError());
    slar::count_launch(), k_mom_t12<<<nmom, 64, 0, s>>>(h.Broot, h.r[4], h.r[5], m34, t12);
    CK(cudaGetLastError());
    dim3 g2((h.r[0] * h.r[1] + 127) / 128, nmom);
    slar::count_launch(), k_mom_bt<<<g2, 128, 0, s>>>(h.B12, h.r[0], h.r[1], h.r[4], t12, Bt);
    CK(cudaGetLastError());
    // X_m = U0 Bt_m (N0 x r1), field_m = X_m U1^T (N0 x N1)
    const int N0 = g.N[0], N1 = g.N[1], r0 = h.r[0], r1 = h.r[1];
    CK(dgemm(0, 0, N0, r1, r0, 1.0, h.U[0], r0, 0, Bt, r1, (long long)r0 * r1, 0.0, c->T1, r1,
             (long long)N0 * r1, nmom, s));
    CK(dgemm(0, 1, N0, N1, r1, 1.0, c->T1, r1, (long long)N0 * r1, h.U[1], r1, 0, 0.0, out, N1,
             (long long)c->NX, nmom, s));
  } else {
    slar::count_launch(), k_mom_root_1d<<<nmom, 64, 0, s>>>(tab, h.r[1], h.Broot, h.r[0], lv, ldr, t12);
    CK(cudaGetLastError());
    dim3 g2((g.N[0] + 127) / 128, nmom);
    slar::count_launch(), k_mom_field_1d<<<g2, 128, 0, s>>>(h.U[0], g.N[0], h.r[0], t12, out, c->NX);
    CK(cudaGetLastError());
  }
  if (with_corr && c->has_corr) {
    dim3 g3((c->NX + 127) / 128, nmom);
    slar::count_launch(), k_corr_moments<<<g3, 128, 0, s>>>(g, tab, c->dC, c->qv, out, nmom);
    CK(cudaGetLastError());
  }
  return SLAR_OK;
}

}  // namespace slar
