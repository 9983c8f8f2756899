// Device functions shared by the entry evaluators (sl_eval.cu: SIMT, FP32/FP64;
// sl_eval_tc.cu: tensor-core transfer-tensor contractions): the characteristic foot, the
// cell weights, spatial and velocity interpolation, the separable LoMaC correction and the
// decoding of an entry index into a grid tuple.  Foot arithmetic uses explicit
// round-to-nearest intrinsics (no FMA contraction) so cell choices are reproducible.
// The FP64 functions take the stencil width S as a template argument: S = 3 is the paper's
// quadratic stencil (Eq. 1d_quadratic_interp_weight), S = 5 the quartic centred Lagrange
// stencil {j-2, ..., j+2} of the higher-order option (remark after Eq. tp_interp); the
// FP32 functions are quadratic only.
#pragma once

#include "common.cuh"

namespace slar {
namespace {

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }

// periodic stencil rows (r0, r0 + 1, ..., r0 + S - 1) mod n, r0 = jf - S/2, for the cell
// index jf (an integer value, |jf| < 1e15): 32-bit arithmetic when jf fits, the 64-bit
// remainder otherwise; the same rows either way (n >= S)
template <int S = 3>
__device__ __forceinline__ void stencil_rows(double jf, int n, int rows[S]) {
  int r0;
  if (fabs(jf) < 1e9) {
    r0 = (int)jf - S / 2;
    if (r0 < 0 || r0 >= n) {
      r0 %= n;
      if (r0 < 0) r0 += n;
    }
  } else {
    long long t = ((long long)jf - S / 2) % n;
    if (t < 0) t += n;
    r0 = (int)t;
  }
  rows[0] = r0;
#pragma unroll
  for (int s = 1; s < S; ++s) rows[s] = rows[s - 1] + 1 == n ? 0 : rows[s - 1] + 1;
}

__device__ __forceinline__ void stencil_rows_f(float jf, int n, int rows[3]) {
  int r0;
  if (fabsf(jf) < 1e9f) {
    r0 = (int)jf - 1;
    if (r0 < 0 || r0 >= n) {
      r0 %= n;
      if (r0 < 0) r0 += n;
    }
  } else {
    long long t = ((long long)jf - 1) % n;
    if (t < 0) t += n;
    r0 = (int)t;
  }
  rows[0] = r0;
  rows[1] = r0 + 1 == n ? 0 : r0 + 1;
  rows[2] = rows[1] + 1 == n ? 0 : rows[1] + 1;
}

// cell and weights of coordinate y in dimension m (oracle: grid.locate and
// grid.stencil_weights): the quadratic weights for S = 3; for S = 5 the quartic Lagrange
// weights L_k(xi) = prod_{m != k} (xi - m) / (k - m), k = -2..2.  RCP: the cell coordinate
// as (y - a) times the FP64 reciprocal of Delta instead of the IEEE quotient (within an ulp
// of it; for the FP32 paths' re-trace, where a dependent FP64 division costs ~440 cycles)
template <int S = 3, bool RCP = false>
__device__ __forceinline__ void cell_weights(const GridDesc& g, int m, double y, int rows[S], double w[S]) {
  static_assert(S == 3 || S == 5, "quadratic or quartic stencils");
  double t = RCP ? dmul(dsub(y, g.lo[m]), g.ih[m]) : __ddiv_rn(dsub(y, g.lo[m]), g.h[m]);
  if (!(fabs(t) < 1e15)) t = 0.0;  // non-finite or absurd feet still index inside the grid
  double jf = floor(t);
  double xi = dsub(dsub(t, jf), 0.5);
  if constexpr (S == 3) {
    double hx = dmul(0.5, xi);
    w[0] = dmul(hx, dsub(xi, 1.0));
    w[1] = dsub(1.0, dmul(xi, xi));
    w[2] = dmul(hx, dadd(xi, 1.0));
  } else {
    const double a = dadd(xi, 2.0), b = dadd(xi, 1.0), e = dsub(xi, 1.0), f = dsub(xi, 2.0);
    const double ab = dmul(a, b), ef = dmul(e, f);
    w[0] = __ddiv_rn(dmul(dmul(b, xi), ef), 24.0);
    w[1] = -__ddiv_rn(dmul(dmul(a, xi), ef), 6.0);
    w[2] = __ddiv_rn(dmul(ab, ef), 4.0);
    w[3] = -__ddiv_rn(dmul(dmul(ab, xi), f), 6.0);
    w[4] = __ddiv_rn(dmul(dmul(ab, xi), e), 24.0);
  }
  stencil_rows<S>(jf, g.N[m], rows);
}

// tensor-product interpolation of a spatial field at point p (dx dims), lexicographic
// stencil order, acc = acc + (w1 w2) v  (oracle: sl.interp_spatial)
template <int S = 3, bool RCP = false>
__device__ double interp_spatial(const GridDesc& g, const double* F, const double* p) {
  int r0[S], r1[S];
  double w0[S], w1[S];
  cell_weights<S, RCP>(g, 0, p[0], r0, w0);
  double acc = 0.0;
  if (g.dx == 1) {
    for (int s = 0; s < S; ++s) acc = dadd(acc, dmul(w0[s], F[r0[s]]));
    return acc;
  }
  cell_weights<S, RCP>(g, 1, p[1], r1, w1);
  const int N1 = g.N[1];
  for (int s0 = 0; s0 < S; ++s0)
    for (int s1 = 0; s1 < S; ++s1)
      acc = dadd(acc, dmul(dmul(w0[s0], w1[s1]), F[r0[s0] * N1 + r1[s1]]));
  return acc;
}

__device__ __forceinline__ double centre(const GridDesc& g, int m, int i) {
  return dadd(g.lo[m], dmul((double)i + 0.5, g.h[m]));
}

// backward foot of the frozen-field characteristic (oracle: sl.trace_feet); the field is
// interpolated with the S-point stencil (RCP: cell coordinates by reciprocals, see
// cell_weights)
template <int S = 3, bool RCP = false>
__device__ void trace_foot(const GridDesc& g, const double* E, double tau, int euler,
                           const int* idx, double* foot) {
  const int dx = g.dx;
  double x[2], v[2];
  for (int m = 0; m < dx; ++m) {
    x[m] = centre(g, m, idx[m]);
    v[m] = centre(g, dx + m, idx[dx + m]);
  }
  const long long NX = g.NX;
  if (euler) {
    for (int m = 0; m < dx; ++m) {
      double e = interp_spatial<S, RCP>(g, E + m * NX, x);
      foot[m] = dsub(x[m], dmul(v[m], tau));
      foot[dx + m] = dadd(v[m], dmul(e, tau));
    }
    return;
  }
  const double h = tau;
  const double half = h / 2.0, two_h = 2.0 * h, sixth = __ddiv_rn(h, 6.0);
  double k1x[2], k1v[2], x2[2], v2[2], k2x[2], k2v[2], x3[2], v3[2], k3x[2], k3v[2];
  for (int m = 0; m < dx; ++m) {
    k1x[m] = -v[m];
    k1v[m] = interp_spatial<S, RCP>(g, E + m * NX, x);
  }
  for (int m = 0; m < dx; ++m) {
    x2[m] = dadd(x[m], dmul(half, k1x[m]));
    v2[m] = dadd(v[m], dmul(half, k1v[m]));
  }
  for (int m = 0; m < dx; ++m) {
    k2x[m] = -v2[m];
    k2v[m] = interp_spatial<S, RCP>(g, E + m * NX, x2);
  }
  for (int m = 0; m < dx; ++m) {
    x3[m] = dadd(dsub(x[m], dmul(h, k1x[m])), dmul(two_h, k2x[m]));
    v3[m] = dadd(dsub(v[m], dmul(h, k1v[m])), dmul(two_h, k2v[m]));
  }
  for (int m = 0; m < dx; ++m) {
    k3x[m] = -v3[m];
    k3v[m] = interp_spatial<S, RCP>(g, E + m * NX, x3);
  }
  for (int m = 0; m < dx; ++m) {
    foot[m] = dadd(x[m], dmul(sixth, dadd(dadd(k1x[m], dmul(4.0, k2x[m])), k3x[m])));
    foot[dx + m] = dadd(v[m], dmul(sixth, dadd(dadd(k1v[m], dmul(4.0, k2v[m])), k3v[m])));
  }
}

// 1D interpolation of a velocity vector (oracle: grid.interp_1d)
template <int S = 3>
__device__ __forceinline__ double interp_1d(const GridDesc& g, int m, const double* vec, double y) {
  int r[S];
  double w[S];
  cell_weights<S>(g, m, y, r, w);
  if constexpr (S == 3) {
    return (w[0] * vec[r[0]] + w[1] * vec[r[1]]) + w[2] * vec[r[2]];
  } else {
    double acc = w[0] * vec[r[0]];
#pragma unroll
    for (int s = 1; s < S; ++s) acc += w[s] * vec[r[s]];
    return acc;
  }
}

// separable LoMaC correction sum_k dC_k(x*) Q_k(v*) at a foot (oracle: sl.correction_at)
template <int S = 3>
__device__ double correction_at(const GridDesc& g, const CorrView& c, const double* foot) {
  const int dx = g.dx, dv = g.dv;
  const long long NX = g.NX;
  const int Nv = g.N[dx];
  double dCi[4];
  for (int k = 0; k < dv + 2; ++k) dCi[k] = interp_spatial<S>(g, c.dC + k * NX, foot);
  double om[2], q1[2], q2[2];
  for (int m = 0; m < dv; ++m) {
    const double y = foot[dx + m];
    om[m] = interp_1d<S>(g, dx + m, c.qv + (0 * dv + m) * Nv, y);
    q1[m] = interp_1d<S>(g, dx + m, c.qv + (1 * dv + m) * Nv, y);
    q2[m] = interp_1d<S>(g, dx + m, c.qv + (2 * dv + m) * Nv, y);
  }
  // terms in the order (0: prod omega), (1+m: q1 at m), (1+dv: q2 at m) for m = 0..dv-1
  double out = 0.0;
  double t = dCi[0];
  for (int m = 0; m < dv; ++m) t *= om[m];
  out += t;
  for (int j = 0; j < dv; ++j) {
    t = dCi[1 + j];
    for (int m = 0; m < dv; ++m) t *= (m == j ? q1[m] : om[m]);
    out += t;
  }
  for (int j = 0; j < dv; ++j) {
    t = dCi[1 + dv];
    for (int m = 0; m < dv; ++m) t *= (m == j ? q2[m] : om[m]);
    out += t;
  }
  return out;
}

__device__ __forceinline__ void decode_tuple(const GridDesc& g, const EvalArgs& a, long long e,
                                             int* idx) {
  if (a.mode == EVAL_TUPLES) {
#pragma unroll
    for (int m = 0; m < 4; ++m)
      if (m < g.d) idx[m] = a.idx[e * g.d + m];
    return;
  }
  // one fibre at *pivot, or fibre e / nper of a block at pivot[e / nper]; every index here
  // is below 2^31 (a launch's entries, a fibre's length, a matricisation's row count), so
  // 32-bit divisions (a 64-bit one is a long software sequence)
  const unsigned eu = (unsigned)e, nper = (unsigned)a.nper;
  const unsigned fib = nper ? eu / nper : 0u;
  const unsigned within = nper ? eu - fib * nper : eu;
  const unsigned piv = (unsigned)a.pivot[fib];
  const unsigned left = (a.mode == EVAL_ROW) ? piv : within;
  const unsigned right = (a.mode == EVAL_ROW) ? within : piv;
  if (g.d == 2) {
    idx[0] = (int)left;
    idx[1] = (int)right;
  } else {
    const unsigned n1 = (unsigned)g.N[1], n3 = (unsigned)g.N[3];
    const unsigned l1 = left / n1, r1 = right / n3;
    idx[0] = (int)l1;
    idx[1] = (int)(left - l1 * n1);
    idx[2] = (int)r1;
    idx[3] = (int)(right - r1 * n3);
  }
}


// ---- FP32 variants (FP32 / BF16 entry paths): the same formulas in single precision.
// Their feet can differ from the FP64 ones by a few FP32 ulps of the displacement.  Where
// that could move an entry to the neighbouring stencil -- its FP32 foot lies within a guard
// of a cell face, and the two quadratic stencils there differ by Delta^3 f''' / 8 -- the foot
// is traced again in FP64 (foot_cells_ft), so both paths interpolate from the same cells.

__device__ __forceinline__ void cell_weights_f(const GridDesc& g, int m, float y, int rows[3], float w[3]) {
  float t = (y - g.lof[m]) * g.ihf[m];
  if (!(fabsf(t) < 1e15f)) t = 0.f;
  const float jf = floorf(t);
  const float xi = t - jf - 0.5f;
  const float hx = 0.5f * xi;
  w[0] = hx * (xi - 1.f);
  w[1] = 1.f - xi * xi;
  w[2] = hx * (xi + 1.f);
  stencil_rows_f(jf, g.N[m], rows);
}

// both (DX) components of a spatial vector field at p, one set of weights; static loops
// over the dimensions keep every small array in registers
template <int DX>
__device__ __forceinline__ void interp_vec_ft(const GridDesc& g, const float* F, const float* p, float* out) {
  int r0[3];
  float w0[3];
  cell_weights_f(g, 0, p[0], r0, w0);
  const long long NX = g.NX;
  if constexpr (DX == 1) {
    out[0] = w0[0] * F[r0[0]] + w0[1] * F[r0[1]] + w0[2] * F[r0[2]];
  } else {
    int r1[3];
    float w1[3];
    cell_weights_f(g, 1, p[1], r1, w1);
    const int N1 = g.N[1];
    float acc[2] = {0.f, 0.f};
#pragma unroll
    for (int s0 = 0; s0 < 3; ++s0)
#pragma unroll
      for (int s1 = 0; s1 < 3; ++s1) {
        const float ww = w0[s0] * w1[s1];
        const long long o = (long long)r0[s0] * N1 + r1[s1];
        acc[0] += ww * F[o];
        acc[1] += ww * F[NX + o];
      }
    out[0] = acc[0];
    out[1] = acc[1];
  }
}

__device__ __forceinline__ float centre_f(const GridDesc& g, int m, int i) {
  return g.lof[m] + ((float)i + 0.5f) * g.hf[m];
}

// backward foot of the frozen-field characteristic (Kutta RK3 or first order), FP32, for
// DX spatial dimensions, as its displacement from the departure cell centre in cells,
// d[m] = (foot_m - centre_m) / Delta_m: the cell and the offset in it then carry FP32 ulps of
// d, not of the absolute cell coordinate (up to N + the box offset in cells).  The velocity
// centres are the FP64 ones rounded once (the x-displacement is tau v), the spatial ones
// only place the field interpolations.
template <int DX>
__device__ __forceinline__ void trace_disp_ft(const GridDesc& g, const float* E, double tau_d, int euler,
                                              const int* idx, float* d) {
  const float tau = (float)tau_d;
  float x[DX], v[DX], e[DX], Dx[DX], Dv[DX];
#pragma unroll
  for (int m = 0; m < DX; ++m) {
    x[m] = centre_f(g, m, idx[m]);
    v[m] = (float)(g.lo[DX + m] + ((double)idx[DX + m] + 0.5) * g.h[DX + m]);
  }
  if (euler) {
    interp_vec_ft<DX>(g, E, x, e);
#pragma unroll
    for (int m = 0; m < DX; ++m) {
      Dx[m] = -v[m] * tau;
      Dv[m] = e[m] * tau;
    }
  } else {
    const float half = 0.5f * tau, two_h = 2.f * tau, sixth = tau / 6.f;
    float k1v[DX], k2x[DX], k2v[DX], k3v[DX], x2[DX], x3[DX], v3[DX];
    interp_vec_ft<DX>(g, E, x, k1v);
#pragma unroll
    for (int m = 0; m < DX; ++m) {
      x2[m] = x[m] - half * v[m];
      k2x[m] = -(v[m] + half * k1v[m]);
    }
    interp_vec_ft<DX>(g, E, x2, k2v);
#pragma unroll
    for (int m = 0; m < DX; ++m) {
      x3[m] = x[m] + tau * v[m] + two_h * k2x[m];
      v3[m] = v[m] - tau * k1v[m] + two_h * k2v[m];
    }
    interp_vec_ft<DX>(g, E, x3, k3v);
#pragma unroll
    for (int m = 0; m < DX; ++m) {
      Dx[m] = sixth * ((-v[m]) + 4.f * k2x[m] + (-v3[m]));
      Dv[m] = sixth * (k1v[m] + 4.f * k2v[m] + k3v[m]);
    }
  }
#pragma unroll
  for (int m = 0; m < DX; ++m) {
    d[m] = Dx[m] * g.ihf[m];
    d[DX + m] = Dv[m] * g.ihf[DX + m];
  }
}

// Both (DX) components of a spatial field at p for the FP32 paths' FP64 re-trace: the same
// IEEE operation sequence per component as interp_spatial<3, true> (so bit-identical
// values), with the cells and weights computed once and the two components' chains side by
// side -- the re-trace's dependent FP64 latency is what a prologue warp waits for.
template <int DX>
__device__ __forceinline__ void interp_vec_rt(const GridDesc& g, const double* E, const double* p, double* out) {
  const long long NX = g.NX;
  int r0[3], r1[3];
  double w0[3], w1[3];
  cell_weights<3, true>(g, 0, p[0], r0, w0);
  if constexpr (DX == 1) {
    double acc = 0.0;
#pragma unroll
    for (int s0 = 0; s0 < 3; ++s0) acc = dadd(acc, dmul(w0[s0], E[r0[s0]]));
    out[0] = acc;
  } else {
    cell_weights<3, true>(g, 1, p[1], r1, w1);
    const int N1 = g.N[1];
    double a0 = 0.0, a1 = 0.0;
#pragma unroll
    for (int s0 = 0; s0 < 3; ++s0)
#pragma unroll
      for (int s1 = 0; s1 < 3; ++s1) {
        const double ww = dmul(w0[s0], w1[s1]);
        const long long o = (long long)r0[s0] * N1 + r1[s1];
        a0 = dadd(a0, dmul(ww, E[o]));
        a1 = dadd(a1, dmul(ww, E[NX + o]));
      }
    out[0] = a0;
    out[1] = a1;
  }
}

// trace_foot<3, true> (the same operations, hence the same foot) with the field
// interpolated by interp_vec_rt
template <int DX>
__device__ __forceinline__ void trace_foot_rt(const GridDesc& g, const double* E, double tau, int euler,
                                              const int* idx, double* foot) {
  double x[DX], v[DX];
#pragma unroll
  for (int m = 0; m < DX; ++m) {
    x[m] = centre(g, m, idx[m]);
    v[m] = centre(g, DX + m, idx[DX + m]);
  }
  if (euler) {
    double e[DX];
    interp_vec_rt<DX>(g, E, x, e);
#pragma unroll
    for (int m = 0; m < DX; ++m) {
      foot[m] = dsub(x[m], dmul(v[m], tau));
      foot[DX + m] = dadd(v[m], dmul(e[m], tau));
    }
    return;
  }
  const double h = tau;
  const double half = h / 2.0, two_h = 2.0 * h, sixth = __ddiv_rn(h, 6.0);
  double k1x[DX], k1v[DX], x2[DX], v2[DX], k2x[DX], k2v[DX], x3[DX], v3[DX], k3x[DX], k3v[DX];
#pragma unroll
  for (int m = 0; m < DX; ++m) k1x[m] = -v[m];
  interp_vec_rt<DX>(g, E, x, k1v);
#pragma unroll
  for (int m = 0; m < DX; ++m) {
    x2[m] = dadd(x[m], dmul(half, k1x[m]));
    v2[m] = dadd(v[m], dmul(half, k1v[m]));
  }
#pragma unroll
  for (int m = 0; m < DX; ++m) k2x[m] = -v2[m];
  interp_vec_rt<DX>(g, E, x2, k2v);
#pragma unroll
  for (int m = 0; m < DX; ++m) {
    x3[m] = dadd(dsub(x[m], dmul(h, k1x[m])), dmul(two_h, k2x[m]));
    v3[m] = dadd(dsub(v[m], dmul(h, k1v[m])), dmul(two_h, k2v[m]));
  }
#pragma unroll
  for (int m = 0; m < DX; ++m) k3x[m] = -v3[m];
  interp_vec_rt<DX>(g, E, x3, k3v);
#pragma unroll
  for (int m = 0; m < DX; ++m) {
    foot[m] = dadd(x[m], dmul(sixth, dadd(dadd(k1x[m], dmul(4.0, k2x[m])), k3x[m])));
    foot[DX + m] = dadd(v[m], dmul(sixth, dadd(dadd(k1v[m], dmul(4.0, k2v[m])), k3v[m])));
  }
}

// Foot, cells and weights of one entry in the FP32 paths (2 DX dimensions): the cells and
// weights of the FP32 foot, unless it lies within a guard of a cell face in some dimension
// m, in which case the entry takes the FP64 foot (E64 given) and its cells and weights
// (rounded to FP32), with the cell coordinates by FP64 reciprocals: within an ulp of the
// FP64 path's quotients, so the same cells except for feet within ~1e-14 cells of a face.  The foot's cell coordinate is idx + 0.5 + d (d from
// trace_disp_ft), so its cell is idx + floor(0.5 + d) and its offset in the cell the
// fraction of u = 0.5 + d.  The FP32 d carries a few ulps of |d| (roundings in the RK3
// combination, the field values and interpolation, the division by Delta) and u half an ulp
// of |u|; the guard is 32 ulps of |d| + 1, several times that.  The velocity field E also
// enters through the intermediate RK3 points, whose FP32 and FP64 positions differ by an ulp
// of x: a field stencil switched there moves the foot by ~tau Delta^3 E''' / Delta, far below
// the guard except in configurations of probability ~1e-9 per entry.  (A dependent FP64
// division costs ~440 cycles on B300 and a warp waits for its slowest lane, so the guard is
// kept tight.)  rows / w: [2 DX][3]; foot: the FP32 foot positions.
template <int DX>
__device__ __forceinline__ void foot_cells_ft(const GridDesc& g, const float* E32, const double* E64, double tau,
                                              int euler, const int* idx, float* foot, int* rows, float* w) {
  constexpr int D = 2 * DX;
  float dsp[D], u[D];
  trace_disp_ft<DX>(g, E32, tau, euler, idx, dsp);
  bool near = false;
#pragma unroll
  for (int m = 0; m < D; ++m) {
    u[m] = 0.5f + dsp[m];
    const float fr = u[m] - floorf(u[m]);
    const float gd = 32.f * 0x1p-23f * (fabsf(dsp[m]) + 1.f);
    near |= !(fr >= gd && fr <= 1.f - gd);   // also catches a non-finite displacement
  }
  if (near && E64) {
    double fd[4];
    trace_foot_rt<DX>(g, E64, tau, euler, idx, fd);
#pragma unroll
    for (int m = 0; m < D; ++m) {
      double wd[3];
      cell_weights<3, true>(g, m, fd[m], rows + 3 * m, wd);
#pragma unroll
      for (int s = 0; s < 3; ++s) w[3 * m + s] = (float)wd[s];
      foot[m] = (float)fd[m];
    }
    return;
  }
#pragma unroll
  for (int m = 0; m < D; ++m) {
    float um = u[m];
    if (!(fabsf(um) < 1e15f)) um = 0.5f;
    const float fu = floorf(um);
    const float xi = (um - fu) - 0.5f;
    const float hx = 0.5f * xi;
    w[3 * m] = hx * (xi - 1.f);
    w[3 * m + 1] = 1.f - xi * xi;
    w[3 * m + 2] = hx * (xi + 1.f);
    stencil_rows_f((float)idx[m] + fu, g.N[m], rows + 3 * m);
    foot[m] = centre_f(g, m, idx[m]) + dsp[m] * g.hf[m];
  }
}

// The same correction from the entry's cells and weights (rows / w: [2 DX][3]), so that it
// interpolates from the cells the HT part used (foot_cells_ft).
template <int DX>
__device__ __forceinline__ float correction_rw_ft(const GridDesc& g, const CorrView& c, const int* rows,
                                                  const float* w) {
  constexpr int DV = DX;
  const long long NX = g.NX;
  const int Nv = g.N[DX];
  float dCi[DV + 2];
  const int* r0 = rows;
  const float* w0 = w;
  const int* r1 = rows + 3;
  const float* w1 = w + 3;
#pragma unroll
  for (int k = 0; k < DV + 2; ++k) {
    const float* F = c.dC32 + k * NX;
    float acc = 0.f;
    if constexpr (DX == 1) {
#pragma unroll
      for (int s0 = 0; s0 < 3; ++s0) acc += w0[s0] * F[r0[s0]];
    } else {
#pragma unroll
      for (int s0 = 0; s0 < 3; ++s0)
#pragma unroll
        for (int s1 = 0; s1 < 3; ++s1) acc += w0[s0] * w1[s1] * F[(long long)r0[s0] * g.N[1] + r1[s1]];
    }
    dCi[k] = acc;
  }
  float om[DV], q1[DV], q2[DV];
#pragma unroll
  for (int m = 0; m < DV; ++m) {
    const int* rv = rows + 3 * (DX + m);
    const float* wv = w + 3 * (DX + m);
    const float* vo = c.qv32 + (0 * DV + m) * Nv;
    const float* v1 = c.qv32 + (1 * DV + m) * Nv;
    const float* v2 = c.qv32 + (2 * DV + m) * Nv;
    om[m] = wv[0] * vo[rv[0]] + wv[1] * vo[rv[1]] + wv[2] * vo[rv[2]];
    q1[m] = wv[0] * v1[rv[0]] + wv[1] * v1[rv[1]] + wv[2] * v1[rv[2]];
    q2[m] = wv[0] * v2[rv[0]] + wv[1] * v2[rv[1]] + wv[2] * v2[rv[2]];
  }
  float out = 0.f, t = dCi[0];
#pragma unroll
  for (int m = 0; m < DV; ++m) t *= om[m];
  out += t;
#pragma unroll
  for (int j = 0; j < DV; ++j) {
    t = dCi[1 + j];
#pragma unroll
    for (int m = 0; m < DV; ++m) t *= (m == j ? q1[m] : om[m]);
    out += t;
  }
#pragma unroll
  for (int j = 0; j < DV; ++j) {
    t = dCi[1 + DV];
#pragma unroll
    for (int m = 0; m < DV; ++m) t *= (m == j ? q2[m] : om[m]);
    out += t;
  }
  return out;
}

}  // namespace
}  // namespace slar
