// The local SL-FD entry evaluator on an HT tensor (Sec. 3.1, Eq. SL_basic_formulation and
// Eq. tp_interp evaluated in HT form).
//
// One CTA evaluates TILE entries:
//   1. foot: backward characteristic of the frozen-field advection through the entry's grid
//      point (Kutta RK3 on dz/ds = (-v, E(x)), E interpolated with the tensor-product
//      quadratic weights; or the first-order foot), then per dimension the cell j and the
//      weights w(xi) of Eq. 1d_quadratic_interp_weight.  FP64 path: explicit round-to-nearest
//      intrinsics (no FMA contraction) so the cell choice reproduces the FP64 oracle's; FP32
//      path: the same formulas in FP32 (B300's FP64 rate per SM sub-partition made the FP64
//      foot the longest phase of a low-rank FP32 evaluation).
//   2. leaf gathers c^(mu) = w . U^(mu)[j-1..j+1, :]  (coalesced row loads, staged in smem);
//      FP64 entries may take the quartic five-point stencil j-2..j+2 instead (g.S = 5: the
//      higher-order option of the remark after Eq. tp_interp, also used for the field at the
//      foot and the correction)
//   3. transfer-tensor contractions c12 = B12 x1 c0 x2 c1, likewise c34: small transfer
//      tensors resident in shared memory (outer products c0 (x) c1 formed on the fly, threads
//      over entries and output ranks); large ones in FP32 as one [TILE x r1] x [r1 x r0] GEMM
//      per output rank followed by the dot with c0 (contract_node_gemm), in FP64 streamed
//      through shared memory in K-chunks.
//   4. root: c12 . Broot . c34 (warp-shuffle reduction)
//   5. separable LoMaC correction (if present) and, for cross-approximation fibres, the
//      residual epilogue out = value - sum_l X[pivot, l] Y[e, l].
// T = double (FP64 path) or float (FP32 path: gathers and contractions in FP32).
#include "common.cuh"
#include "eval_device.cuh"

namespace slar {
namespace {

constexpr int NTHREADS = 256;
constexpr int KC = 32;          // K-chunk of the transfer-tensor contraction
constexpr int PSTRIDE = 65;     // padded row of the staged B chunk (p <= 64)

// Transfer tensors small enough for this byte budget are staged whole in shared memory
// ([k][p], k = (a, b)) by the warps that do not trace feet, while the feet are traced;
// larger ones stream through a [KC][PSTRIDE] chunk buffer.
constexpr int RES_BYTES = 48 * 1024;

template <typename T>
__host__ __device__ __forceinline__ bool b_resident(int d, int r0, int r1, int r2, int r3, int r12, int r34) {
  return d == 4 && (long long)(r0 * r1 * r12 + r2 * r3 * r34) * (long long)sizeof(T) <= RES_BYTES;
}

// with resident transfer tensors, a root matrix of at most ROOT_RES_BYTES is staged too, so
// the root contraction reads shared memory instead of waiting on global loads
constexpr int ROOT_RES_BYTES = 8 * 1024;

template <typename T>
__host__ __device__ __forceinline__ bool root_resident(int d, int r0, int r1, int r2, int r3, int r12, int r34) {
  return b_resident<T>(d, r0, r1, r2, r3, r12, r34) && (long long)r12 * r34 * (long long)sizeof(T) <= ROOT_RES_BYTES;
}

// c_out[t][p] = sum_{a,b} ca[t][a] cb[t][b] sB[(a,b)][p] with the whole transfer tensor resident
template <typename T, int TILE>
__device__ void contract_node_res(const T* __restrict__ ca, int ra, const T* __restrict__ cb, int rb,
                                  const T* __restrict__ sBn, int rp, T* __restrict__ cout, int nT) {
  constexpr int TPT = TILE / 8;
  const int tid = threadIdx.x;
  const int tg = tid >> 5, lane = tid & 31;
  T acc[TPT][2];
#pragma unroll
  for (int i = 0; i < TPT; ++i) acc[i][0] = acc[i][1] = T(0);
  int kk = 0;
  for (int a = 0; a < ra; ++a) {
    T xa[TPT];
#pragma unroll
    for (int i = 0; i < TPT; ++i) xa[i] = ca[(tg * TPT + i) * ra + a];
    for (int b = 0; b < rb; ++b, ++kk) {
      const T b0 = (lane < rp) ? sBn[kk * rp + lane] : T(0);
      const T b1 = (lane + 32 < rp) ? sBn[kk * rp + lane + 32] : T(0);
#pragma unroll
      for (int i = 0; i < TPT; ++i) {
        const T x = xa[i] * cb[(tg * TPT + i) * rb + b];
        acc[i][0] += x * b0;
        acc[i][1] += x * b1;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < TPT; ++i) {
    const int t = tg * TPT + i;
    if (t < nT) {
      if (lane < rp) cout[t * rp + lane] = acc[i][0];
      if (lane + 32 < rp) cout[t * rp + lane + 32] = acc[i][1];
    }
  }
}

// The same contraction for small output ranks (rp <= PPER * NTHREADS / TILE): thread
// (t, q) with TPE = NTHREADS / TILE threads per entry accumulates p = q, q + TPE, ...
// (PPER outputs).  Lanes over p, as above, would leave most of a warp idle at the ranks of
// weakly perturbed runs (4-20); here every lane works and each product ca cb is formed once
// per thread for its PPER outputs.
template <typename T, int TILE, int PPER>
__device__ void contract_node_res_small(const T* __restrict__ ca, int ra, const T* __restrict__ cb, int rb,
                                        const T* __restrict__ sBn, int rp, T* __restrict__ cout, int nT) {
  constexpr int TPE = NTHREADS / TILE;
  const int t = threadIdx.x / TPE, q = threadIdx.x - t * TPE;
  T acc[PPER];
#pragma unroll
  for (int j = 0; j < PPER; ++j) acc[j] = T(0);
  const T* cat = ca + t * ra;
  const T* cbt = cb + t * rb;
  int kk = 0;
  for (int a = 0; a < ra; ++a) {
    const T xa = cat[a];
    for (int b = 0; b < rb; ++b, ++kk) {
      const T x = xa * cbt[b];
      const T* Bk = sBn + kk * rp;
#pragma unroll
      for (int j = 0; j < PPER; ++j) {
        const int p = q + j * TPE;
        if (p < rp) acc[j] += x * Bk[p];
      }
    }
  }
  if (t < nT) {
#pragma unroll
    for (int j = 0; j < PPER; ++j) {
      const int p = q + j * TPE;
      if (p < rp) cout[t * rp + p] = acc[j];
    }
  }
}

template <typename T, int TILE>
__device__ __forceinline__ void contract_res(const T* ca, int ra, const T* cb, int rb, const T* sBn, int rp,
                                             T* cout, int nT) {
  constexpr int TPE = NTHREADS / TILE;
  if (rp <= 2 * TPE) contract_node_res_small<T, TILE, 2>(ca, ra, cb, rb, sBn, rp, cout, nT);
  else if (rp <= 4 * TPE) contract_node_res_small<T, TILE, 4>(ca, ra, cb, rb, sBn, rp, cout, nT);
  else contract_node_res<T, TILE>(ca, ra, cb, rb, sBn, rp, cout, nT);
}

// c_out[t][p] = sum_{a,b} ca[t][a] cb[t][b] B[p][a][b]   for t < nT, p < rp
template <typename T, int TILE>
__device__ void contract_node(const T* __restrict__ ca, int ra, const T* __restrict__ cb, int rb,
                              const T* __restrict__ B, int rp, T* __restrict__ cout, T* sB, int nT) {
  constexpr int TPT = TILE / 8;  // entries per thread
  const int tid = threadIdx.x;
  const int tg = tid >> 5, lane = tid & 31;
  const int K = ra * rb;
  T acc[TPT][2];
#pragma unroll
  for (int i = 0; i < TPT; ++i) acc[i][0] = acc[i][1] = T(0);
  for (int k0 = 0; k0 < K; k0 += KC) {
    const int kc = min(KC, K - k0);
    __syncthreads();
    for (int it = tid; it < kc * rp; it += NTHREADS) {
      const int p = it / kc, kk = it - p * kc;
      sB[kk * PSTRIDE + p] = B[(long long)p * K + k0 + kk];
    }
    __syncthreads();
    int a = k0 / rb, b = k0 - a * rb;
    for (int kk = 0; kk < kc; ++kk) {
      const T b0 = (lane < rp) ? sB[kk * PSTRIDE + lane] : T(0);
      const T b1 = (lane + 32 < rp) ? sB[kk * PSTRIDE + lane + 32] : T(0);
#pragma unroll
      for (int i = 0; i < TPT; ++i) {
        const int t = tg * TPT + i;
        const T x = ca[t * ra + a] * cb[t * rb + b];
        acc[i][0] += x * b0;
        acc[i][1] += x * b1;
      }
      if (++b == rb) { b = 0; ++a; }
    }
  }
#pragma unroll
  for (int i = 0; i < TPT; ++i) {
    const int t = tg * TPT + i;
    if (t < nT) {
      if (lane < rp) cout[t * rp + lane] = acc[i][0];
      if (lane + 32 < rp) cout[t * rp + lane + 32] = acc[i][1];
    }
  }
}

// FP32 contraction for transfer tensors too large to stay resident (ranks above ~22): for
// each output rank p, T[t][a] = sum_b cb[t][b] B[p][a][b] is a [TILE x rb] x [rb x ra] GEMM,
// register-tiled as 4 a x EPT entries per thread (16 a-groups x 16 entry groups), with cb
// staged transposed so that every k-step is two vector shared loads for 4 EPT FMAs; then
// c_out[t][p] = sum_a ca[t][a] T[t][a] (the thread's ca values stay in registers across p)
// reduced over the 16 a-groups of a half-warp.  B[p] (ra x rb, contiguous) is loaded into
// registers while p - 1 is computed and stored transposed into shared memory.
constexpr int GEMM_LDB = 68;   // row stride (floats) of the staged B[p]^T: a < 64, 16-byte rows

__host__ __device__ __forceinline__ int gemm_ldt(int tile) { return tile + 4; }

__host__ __device__ __forceinline__ size_t gemm_smem_floats(int tile, int rbmax) {
  return (size_t)rbmax * gemm_ldt(tile) + (size_t)rbmax * GEMM_LDB;
}

template <int TILE>
__device__ void contract_node_gemm(const float* __restrict__ ca, int ra, const float* __restrict__ cb, int rb,
                                   const float* __restrict__ B, int rp, float* __restrict__ cout, int nT,
                                   float* sbuf) {
  constexpr int EPT = TILE / 16;
  constexpr int LDT = TILE + 4;
  const int tid = threadIdx.x;
  const int eg = tid >> 4, ag = tid & 15;
  float* sCt = sbuf;                 // [rb][LDT]: cb transposed
  float* sBt = sbuf + rb * LDT;      // [rb][GEMM_LDB]: B[p] transposed, zero beyond ra
  __syncthreads();                   // the previous user of sbuf is done
  for (int it = tid; it < TILE * rb; it += NTHREADS) {
    const int t = it / rb, b = it - t * rb;
    sCt[b * LDT + t] = cb[it];
  }
  for (int it = tid; it < rb * GEMM_LDB; it += NTHREADS) sBt[it] = 0.f;
  float c1[EPT][4];
#pragma unroll
  for (int i = 0; i < EPT; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int a = ag * 4 + j;
      c1[i][j] = a < ra ? ca[(eg * EPT + i) * ra + a] : 0.f;
    }
  const int nab = ra * rb;           // <= 4096: at most 16 elements per thread
  float pre[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int it = tid + j * NTHREADS;
    pre[j] = it < nab ? __ldg(B + it) : 0.f;
  }
  for (int p = 0; p < rp; ++p) {
    __syncthreads();                 // staging of sCt / the previous p's reads of sBt are done
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int it = tid + j * NTHREADS;
      if (it < nab) {
        const int a = it / rb, b = it - a * rb;
        sBt[b * GEMM_LDB + a] = pre[j];
      }
    }
    __syncthreads();
    if (p + 1 < rp) {
      const float* Bn = B + (long long)(p + 1) * nab;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int it = tid + j * NTHREADS;
        pre[j] = it < nab ? __ldg(Bn + it) : 0.f;
      }
    }
    float acc[EPT][4];
#pragma unroll
    for (int i = 0; i < EPT; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    const float* cp = sCt + eg * EPT;
    const float* bp = sBt + ag * 4;
#pragma unroll 4
    for (int b = 0; b < rb; ++b) {
      const float4 bv = *reinterpret_cast<const float4*>(bp + b * GEMM_LDB);
      float cv[EPT];
      if constexpr (EPT == 4) {
        const float4 t4 = *reinterpret_cast<const float4*>(cp + b * LDT);
        cv[0] = t4.x; cv[1] = t4.y; cv[2] = t4.z; cv[3] = t4.w;
      } else if constexpr (EPT == 2) {
        const float2 t2 = *reinterpret_cast<const float2*>(cp + b * LDT);
        cv[0] = t2.x; cv[1] = t2.y;
      } else {
        cv[0] = cp[b * LDT];
      }
#pragma unroll
      for (int i = 0; i < EPT; ++i) {
        acc[i][0] = fmaf(cv[i], bv.x, acc[i][0]);
        acc[i][1] = fmaf(cv[i], bv.y, acc[i][1]);
        acc[i][2] = fmaf(cv[i], bv.z, acc[i][2]);
        acc[i][3] = fmaf(cv[i], bv.w, acc[i][3]);
      }
    }
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      float s = (c1[i][0] * acc[i][0] + c1[i][1] * acc[i][1]) + (c1[i][2] * acc[i][2] + c1[i][3] * acc[i][3]);
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const int t = eg * EPT + i;
      if (ag == 0 && t < nT) cout[t * rp + p] = s;
    }
  }
}

// FP64 foot, cells and weights of entry e with the S-point stencil: foot[4], rows / w [4][S]
// (at_grid: the grid point itself, weight 1 on its own row)
template <int S>
__device__ __forceinline__ void feet_cells64(const GridDesc& g, const EvalArgs& a, long long e, int at_grid,
                                             double* foot, int* rows, double* w) {
  int idx[4];
  decode_tuple(g, a, e, idx);
  double ft[4];
  if (at_grid) {
    for (int m = 0; m < g.d; ++m) ft[m] = centre(g, m, idx[m]);
  } else {
    trace_foot<S>(g, a.E, a.tau, a.foot_euler, idx, ft);
  }
  for (int m = 0; m < g.d; ++m) {
    int r[S];
    double ww[S];
    if (at_grid) {
#pragma unroll
      for (int s = 0; s < S; ++s) {
        r[s] = idx[m];
        ww[s] = s == S / 2 ? 1.0 : 0.0;
      }
    } else {
      cell_weights<S>(g, m, ft[m], r, ww);
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      rows[m * S + s] = r[s];
      w[m * S + s] = ww[s];
    }
    foot[m] = ft[m];
  }
}

template <typename T, int TILE>
__device__ __forceinline__ void sl_eval_body(const GridDesc& g, const HTView<T>& ht,
                                             const CorrView& corr, EvalArgs a, int at_grid) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if ((a.done && *a.done) || (a.skip && *a.skip)) return;
  if (a.kidx) {
    const int kk = *a.kidx;
    a.pivot += kk;
    a.kterms = kk;
    a.out += kk * a.out_stride;
  }
  const long long e0 = (long long)blockIdx.x * TILE;
  // a block of fibres evaluates only its *nact active fibres
  const long long n_act = a.nact ? min(a.n, (long long)(*a.nact) * a.nper) : a.n;
  if (e0 >= n_act) return;
  const int nT = (int)min((long long)TILE, n_act - e0);
  const int tid = threadIdx.x;
  const int d = g.d;

  const int S = g.S;                                           // stencil points (3 or 5)
  double* sfoot = reinterpret_cast<double*>(smem_raw);        // TILE*4
  double* sw = sfoot + TILE * 4;                               // TILE*4*S
  double* sval = sw + TILE * 4 * S;                            // TILE
  double* sres = sval + TILE;                                  // TILE residual sums
  int* srow = reinterpret_cast<int*>(sres + TILE);             // TILE*4*S
  T* sfootT = reinterpret_cast<T*>(sfoot);   // the feet and weights in the entry type (FP32
  T* swT = reinterpret_cast<T*>(sw);         // paths: no FP64 conversions in the gathers)
  T* sc = reinterpret_cast<T*>(srow + TILE * 4 * S);           // leaves
  T* sc_mu[4];
  {
    T* p = sc;
    for (int m = 0; m < d; ++m) { sc_mu[m] = p; p += TILE * ht.r[m]; }
    sc = p;
  }
  T* sc12 = sc;
  T* sc34 = sc12 + (d == 4 ? TILE * ht.r12 : 0);
  T* sB = sc34 + (d == 4 ? TILE * ht.r34 : 0);
  const bool resident = b_resident<T>(d, ht.r[0], ht.r[1], ht.r[2], ht.r[3], ht.r12, ht.r34);
  const bool root_res = root_resident<T>(d, ht.r[0], ht.r[1], ht.r[2], ht.r[3], ht.r12, ht.r34);
  const int K12 = ht.r[0] * ht.r[1];
  const int nB = resident ? K12 * ht.r12 + ht.r[2] * ht.r[3] * ht.r34 : 0;
  T* sRoot = sB + nB;   // [r12][r34] when root_res

  // 0. work that does not need the feet, done by the other warps while they are traced:
  // the cross-approximation residual sum_l X[pivot, l] Y[e, l] of each entry, and the
  // resident transfer tensors
  if (tid >= TILE) {
    if (a.X && tid < 2 * TILE) {
      const int t = tid - TILE;
      double r = 0.0;
      if (t < nT) {
        // residual of fibre element `e` against the k previous terms: X at the fibre's pivot,
        // Y at the element's position along the fibre
        const unsigned et = (unsigned)(e0 + t), nper = (unsigned)a.nper;   // below 2^31: 32-bit division
        const unsigned fib = nper ? et / nper : 0u;
        const long long piv = (long long)a.pivot[fib];
        const long long e = (long long)(nper ? et - fib * nper : et);
        const int k = a.kterms;
        int l = 0;
        for (; l + 4 <= k; l += 4) {
          const double y0 = a.Y[e + l * a.ldY], y1 = a.Y[e + (l + 1) * a.ldY];
          const double y2 = a.Y[e + (l + 2) * a.ldY], y3 = a.Y[e + (l + 3) * a.ldY];
          r += a.X[piv + l * a.ldX] * y0;
          r += a.X[piv + (l + 1) * a.ldX] * y1;
          r += a.X[piv + (l + 2) * a.ldX] * y2;
          r += a.X[piv + (l + 3) * a.ldX] * y3;
        }
        for (; l < k; ++l) r += a.X[piv + l * a.ldX] * a.Y[e + l * a.ldY];
      }
      sres[t] = r;
    }
    if (resident) {
      const int n12 = K12 * ht.r12, n34 = ht.r[2] * ht.r[3] * ht.r34;
      const int nroot = root_res ? ht.r12 * ht.r34 : 0;
      for (int it = tid - TILE; it < n12 + n34 + nroot; it += NTHREADS - TILE) {
        if (it < n12) {
          const int p = it / K12, k = it - p * K12;
          sB[k * ht.r12 + p] = ht.B12[it];
        } else if (it < n12 + n34) {
          const int j = it - n12, K34 = ht.r[2] * ht.r[3];
          const int p = j / K34, k = j - p * K34;
          sB[n12 + k * ht.r34 + p] = ht.B34[j];
        } else {
          sRoot[it - n12 - n34] = ht.Broot[it - n12 - n34];
        }
      }
    }
  }

  // 1. feet and weights (FP32 entries: traced in FP32, see eval_device.cuh)
  if constexpr (sizeof(T) == 4) {
    if (tid < nT) {
      int idx[4];
      decode_tuple(g, a, e0 + tid, idx);
      float foot[4] = {0.f, 0.f, 0.f, 0.f};
      int r[12];
      float w[12];
      if (at_grid) {
#pragma unroll
        for (int m = 0; m < 4; ++m)
          if (m < d) {
            foot[m] = centre_f(g, m, idx[m]);
            r[3 * m] = r[3 * m + 1] = r[3 * m + 2] = idx[m];
            w[3 * m] = 0.f; w[3 * m + 1] = 1.f; w[3 * m + 2] = 0.f;
          }
      } else if (g.dx == 2) {
        foot_cells_ft<2>(g, a.E32, a.E, a.tau, a.foot_euler, idx, foot, r, w);
      } else {
        foot_cells_ft<1>(g, a.E32, a.E, a.tau, a.foot_euler, idx, foot, r, w);
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        if (m >= d) break;
        for (int s = 0; s < 3; ++s) {
          srow[(tid * 4 + m) * 3 + s] = r[3 * m + s];
          swT[(tid * 4 + m) * 3 + s] = w[3 * m + s];
        }
        sfootT[tid * 4 + m] = foot[m];
      }
    }
  } else if (tid < nT) {
    if (S == 5)
      feet_cells64<5>(g, a, e0 + tid, at_grid, sfoot + tid * 4, srow + tid * 4 * 5, sw + tid * 4 * 5);
    else
      feet_cells64<3>(g, a, e0 + tid, at_grid, sfoot + tid * 4, srow + tid * 4 * 3, sw + tid * 4 * 3);
  }
  __syncthreads();

  // 2. leaf gathers
  for (int m = 0; m < d; ++m) {
    const int r = ht.r[m];
    const T* U = ht.U[m];
    T* c = sc_mu[m];
    for (int it = tid; it < TILE * r; it += NTHREADS) {
      const int t = it / r, q = it - t * r;
      T val = T(0);
      if (t < nT) {
        const int* rr = srow + (t * 4 + m) * S;
        const T* ww = swT + (t * 4 + m) * S;
        val = ww[0] * U[(long long)rr[0] * r + q] + ww[1] * U[(long long)rr[1] * r + q] +
              ww[2] * U[(long long)rr[2] * r + q];
        if (S == 5) val += ww[3] * U[(long long)rr[3] * r + q] + ww[4] * U[(long long)rr[4] * r + q];
      }
      c[it] = val;
    }
  }
  __syncthreads();

  // 3. transfer tensors
  const T* left;
  const T* right;
  int rl, rr;
  if (d == 4) {
    if (resident) {
      contract_res<T, TILE>(sc_mu[0], ht.r[0], sc_mu[1], ht.r[1], sB, ht.r12, sc12, nT);
      contract_res<T, TILE>(sc_mu[2], ht.r[2], sc_mu[3], ht.r[3], sB + K12 * ht.r12, ht.r34, sc34, nT);
    } else if constexpr (sizeof(T) == 4) {
      contract_node_gemm<TILE>(sc_mu[0], ht.r[0], sc_mu[1], ht.r[1], ht.B12, ht.r12, sc12, nT, sB);
      contract_node_gemm<TILE>(sc_mu[2], ht.r[2], sc_mu[3], ht.r[3], ht.B34, ht.r34, sc34, nT, sB);
    } else {
      contract_node<T, TILE>(sc_mu[0], ht.r[0], sc_mu[1], ht.r[1], ht.B12, ht.r12, sc12, sB, nT);
      contract_node<T, TILE>(sc_mu[2], ht.r[2], sc_mu[3], ht.r[3], ht.B34, ht.r34, sc34, sB, nT);
    }
    left = sc12; right = sc34; rl = ht.r12; rr = ht.r34;
  } else {
    left = sc_mu[0]; right = sc_mu[1]; rl = ht.r[0]; rr = ht.r[1];
  }
  __syncthreads();

  // 4. root: sum_p left[t][p] sum_q Broot[p][q] right[t][q]
  {
    constexpr int TPE = NTHREADS / TILE;  // threads per entry
    const int t = tid / TPE, sub = tid - t * TPE;
    T acc = T(0);
    const T* Broot = (d == 4 && root_res) ? sRoot : ht.Broot;
    if (t < nT) {
      for (int p = sub; p < rl; p += TPE) {
        T s = T(0);
        const T* Bp = Broot + (long long)p * rr;
        for (int q = 0; q < rr; ++q) s += Bp[q] * right[t * rr + q];
        acc += left[t * rl + p] * s;
      }
    }
#pragma unroll
    for (int off = TPE / 2; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off, TPE);
    if (sub == 0 && t < TILE) sval[t] = (double)acc;
  }
  __syncthreads();

  // 5. correction and residual epilogue
  if (tid < nT) {
    double val = sval[tid];
    if (corr.has) {
      if constexpr (sizeof(T) == 4) {
        // from the cells the HT part used (foot_cells_ft)
        const int* rr = srow + tid * 12;
        const float* ww = reinterpret_cast<const float*>(swT) + tid * 12;
        val += (double)(d == 4 ? correction_rw_ft<2>(g, corr, rr, ww) : correction_rw_ft<1>(g, corr, rr, ww));
      } else {
        val += S == 5 ? correction_at<5>(g, corr, sfoot + tid * 4) : correction_at<3>(g, corr, sfoot + tid * 4);
      }
    }
    const long long e = e0 + tid;
    if (a.X) val -= sres[tid];
    a.out[e] = val;
  }
}

template <typename T, int TILE>
__global__ void __launch_bounds__(NTHREADS)
k_sl_eval(GridDesc g, HTView<T> ht, CorrView corr, EvalArgs a, int at_grid) {
  sl_eval_body<T, TILE>(g, ht, corr, a, at_grid);
}

template <typename T, int TILE>
__global__ void __launch_bounds__(NTHREADS)
k_sl_eval_dev(GridDesc g, const EvalParams<T>* __restrict__ P, EvalArgs a) {
  const EvalParams<T> q = *P;
  a.tau = q.tau;
  a.E = q.E;
  a.E32 = q.E32;
  a.foot_euler = q.foot_euler;
  sl_eval_body<T, TILE>(g, q.ht, q.corr, a, 0);
}

template <typename T, int TILE>
size_t smem_bytes(const GridDesc& g, const HTView<T>& ht) {
  const int ns = TILE * 4 * g.S;   // stencil rows and weights
  size_t b = sizeof(double) * (TILE * 4 + ns + TILE + TILE) + sizeof(int) * ns;
  int rs = 0;
  for (int m = 0; m < g.d; ++m) rs += ht.r[m];
  if (g.d == 4) rs += ht.r12 + ht.r34;
  size_t nb = 0;
  if (g.d == 4) {
    const int rbmax = ht.r[1] > ht.r[3] ? ht.r[1] : ht.r[3];
    nb = b_resident<T>(g.d, ht.r[0], ht.r[1], ht.r[2], ht.r[3], ht.r12, ht.r34)
             ? (size_t)ht.r[0] * ht.r[1] * ht.r12 + (size_t)ht.r[2] * ht.r[3] * ht.r34
             : (sizeof(T) == 4 ? gemm_smem_floats(TILE, rbmax) : (size_t)KC * PSTRIDE);
    if (root_resident<T>(g.d, ht.r[0], ht.r[1], ht.r[2], ht.r[3], ht.r12, ht.r34)) nb += (size_t)ht.r12 * ht.r34;
  }
  b += sizeof(T) * ((size_t)TILE * rs + nb);
  return (b + 15) & ~size_t(15);
}

template <typename T, int TILE>
cudaError_t launch_tile(const GridDesc& g, const HTView<T>& ht, const CorrView& corr, const EvalArgs& a,
                        int at_grid, cudaStream_t s) {
  const size_t sm = smem_bytes<T, TILE>(g, ht);
  const long long blocks = (a.n + TILE - 1) / TILE;
  slar::count_launch(), k_sl_eval<T, TILE><<<(unsigned)blocks, NTHREADS, sm, s>>>(g, ht, corr, a, at_grid);
  return cudaGetLastError();
}

template <typename T, int TILE>
cudaError_t launch_tile_dev(const GridDesc& g, const EvalParams<T>* P, const EvalArgs& a, size_t sm,
                            cudaStream_t s) {
  const long long blocks = (a.n + TILE - 1) / TILE;
  slar::count_launch(), k_sl_eval_dev<T, TILE><<<(unsigned)blocks, NTHREADS, sm, s>>>(g, P, a);
  return cudaGetLastError();
}

constexpr int kEvalSmemMax = 200 * 1024;   // opt-in dynamic shared memory of the evaluators

template <typename T, int TILE>
cudaError_t set_attrs_tile() {
  const int mx = kEvalSmemMax;
  cudaError_t e = cudaFuncSetAttribute(k_sl_eval<T, TILE>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sl_eval_dev<T, TILE>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  return e;
}

}  // namespace

bool eval_tile_ok(int tile) { return tile == 16 || tile == 32 || tile == 64; }

template <typename T>
size_t sl_eval_smem(const GridDesc& g, const int* r6, int tile);

// the largest tile <= `tile` (16, 32, 64) whose shared memory fits the evaluator's opt-in
// limit at these ranks (FP64 at rank 64 with tile 64 does not)
template <typename T>
int sl_eval_fit_tile(const GridDesc& g, const int* r6, int tile) {
  while (tile > 16 && sl_eval_smem<T>(g, r6, tile) > (size_t)kEvalSmemMax) tile /= 2;
  return tile;
}
template int sl_eval_fit_tile<double>(const GridDesc&, const int*, int);
template int sl_eval_fit_tile<float>(const GridDesc&, const int*, int);

template <typename T>
cudaError_t launch_sl_eval(const GridDesc& g, const HTView<T>& ht, const CorrView& corr,
                           const EvalArgs& a, int at_grid, cudaStream_t s, int tile) {
  if (a.n <= 0) return cudaSuccess;
  switch (tile) {
    case 16: return launch_tile<T, 16>(g, ht, corr, a, at_grid, s);
    case 64: return launch_tile<T, 64>(g, ht, corr, a, at_grid, s);
    default: return launch_tile<T, 32>(g, ht, corr, a, at_grid, s);
  }
}

cudaError_t sl_eval_init_attrs() {
  cudaError_t e = set_attrs_tile<double, 16>();
  if (e == cudaSuccess) e = set_attrs_tile<double, 32>();
  if (e == cudaSuccess) e = set_attrs_tile<double, 64>();
  if (e == cudaSuccess) e = set_attrs_tile<float, 16>();
  if (e == cudaSuccess) e = set_attrs_tile<float, 32>();
  if (e == cudaSuccess) e = set_attrs_tile<float, 64>();
  return e;
}

template <typename T>
size_t sl_eval_smem(const GridDesc& g, const int* r6, int tile) {
  HTView<T> v{};
  for (int m = 0; m < 4; ++m) v.r[m] = r6[m];
  v.r12 = r6[4];
  v.r34 = r6[5];
  switch (tile) {
    case 16: return smem_bytes<T, 16>(g, v);
    case 64: return smem_bytes<T, 64>(g, v);
    default: return smem_bytes<T, 32>(g, v);
  }
}

template <typename T>
cudaError_t launch_sl_eval_dev(const GridDesc& g, const EvalParams<T>* P, const EvalArgs& a,
                               size_t sm, cudaStream_t s, int tile) {
  switch (tile) {
    case 16: return launch_tile_dev<T, 16>(g, P, a, sm, s);
    case 64: return launch_tile_dev<T, 64>(g, P, a, sm, s);
    default: return launch_tile_dev<T, 32>(g, P, a, sm, s);
  }
}

template size_t sl_eval_smem<double>(const GridDesc&, const int*, int);
template size_t sl_eval_smem<float>(const GridDesc&, const int*, int);
template cudaError_t launch_sl_eval_dev<double>(const GridDesc&, const EvalParams<double>*,
                                                const EvalArgs&, size_t, cudaStream_t, int);
template cudaError_t launch_sl_eval_dev<float>(const GridDesc&, const EvalParams<float>*,
                                               const EvalArgs&, size_t, cudaStream_t, int);
template cudaError_t launch_sl_eval<double>(const GridDesc&, const HTView<double>&,
                                            const CorrView&, const EvalArgs&, int, cudaStream_t, int);
template cudaError_t launch_sl_eval<float>(const GridDesc&, const HTView<float>&,
                                           const CorrView&, const EvalArgs&, int, cudaStream_t, int);

}  // namespace slar
