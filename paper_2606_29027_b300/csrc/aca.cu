// Cross approximation of the SL-updated tensor (the HTACA step of SLAR, Sec. 3.1): the
// matricisation A = F_(x | v) is approximated by U V^T from sampled row and column fibres,
// with partial pivoting; then the exact HT embedding and the HSVD truncation.
//
// Reading of the paper (which defers HTACA to earlier work): partially pivoted ACA on the
// root split, start row 0, stop when ||u_k|| ||v_k|| <= eps ||A_k||_F (running estimate)
// and the residual on q = min(8, M1) fixed check rows (golden-ratio sequence
// floor(frac(c g) M1)) confirms it, (M1/q) sum_c ||R_c||^2 <= eps^2 ||A_k||_F^2, or k = cap;
// when the check fails the next row pivot is the unused check row of largest residual.
// Arg-max ties within a relative 1e-10 go to the lowest index.
//
// Every step runs on the device with no host round trip: the entry evaluator samples the
// residual row (fused residual epilogue), one CTA picks the column pivot and scales v_k,
// the evaluator samples the residual column into u_k, a grid kernel forms the dot products
// of the norm estimate, and one CTA updates the estimate, tests the stop rule and picks the
// next row pivot.  A device flag makes the remaining launches of a stopped approximation
// exit immediately; the host reads the final rank once.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "context.cuh"

namespace slar {
namespace {

constexpr int PIV_THREADS = 1024;
constexpr int ACA_UNROLL = 2;      // pivot steps per iteration of the captured WHILE loop
constexpr int DOT_SEG = 256;      // entries per dot-product block (= its thread count)
constexpr double TIE_RTOL = 1e-10;
// a residual row whose largest unused entry is at most max(NOISE_RTOL, eps / 100) of the first
// pivot is negligible: below eps / 100 a pivot only resolves structure beneath the requested
// accuracy while multiplying rounding errors by 1 / |pivot|, and at NOISE_RTOL the row is
// rounding noise (a repeat of a crossed row, or data reproduced exactly).  No pivot is taken
// in it; it counts as a vanishing term for the stop test.
constexpr double NOISE_RTOL = 1e-14;

// |a| as an order key on the integer pipe: for non-negative doubles the IEEE-754 bit pattern
// orders like the value, so the scans below compare 64-bit integers instead of issuing FP64
// compares (B300 retires about two FP64 operations per clock per SM).  Used entries and NaNs
// get key -1, as fmax / >= ignore NaNs.
__device__ __forceinline__ long long abs_key(double x) {
  const long long b = __double_as_longlong(x) & 0x7fffffffffffffffLL;
  return b > 0x7ff0000000000000LL ? -1LL : b;
}

__device__ __forceinline__ long long warp_max_ll(long long v) {
  for (int o = 16; o > 0; o >>= 1) {
    const long long u = __shfl_down_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  return v;
}

__device__ void block_argmax_tie(const double* a, int n, const unsigned char* used, int* out_idx,
                                 double* out_max) {
  // two passes: global max of |a| over unused, then the lowest index within the tie band
  __shared__ long long wmax[32];
  __shared__ int widx[32];
  const int nthr = blockDim.x, nw = blockDim.x >> 5;
  __shared__ long long top_s;
  const int tid = threadIdx.x;
  long long m = -1;
  for (int i = tid; i < n; i += nthr) {
    const long long k = used[i] ? -1LL : abs_key(a[i]);
    m = k > m ? k : m;
  }
  m = warp_max_ll(m);
  if ((tid & 31) == 0) wmax[tid >> 5] = m;
  __syncthreads();
  if (tid == 0) {
    long long t = -1;
    for (int w = 0; w < nw; ++w) t = wmax[w] > t ? wmax[w] : t;
    top_s = t;
  }
  __syncthreads();
  const long long topk = top_s;
  const double top = topk >= 0 ? __longlong_as_double(topk) : -1.0;
  const long long thrk = topk >= 0 ? __double_as_longlong(top * (1.0 - TIE_RTOL)) : 0x7fffffffffffffffLL;
  int best = 0x7fffffff;
  if (topk >= 0)
    for (int i = tid; i < n; i += nthr)
      if (i < best && !used[i] && abs_key(a[i]) >= thrk) best = i;
  for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_down_sync(0xffffffffu, best, o));
  if ((tid & 31) == 0) widx[tid >> 5] = best;
  __syncthreads();
  if (tid == 0) {
    int b = 0x7fffffff;
    for (int w = 0; w < nw; ++w) b = min(b, widx[w]);
    *out_idx = (topk >= 0 && b != 0x7fffffff) ? b : -1;
    *out_max = top;
  }
  __syncthreads();
}

// The same arg-max with tie band as block_argmax_tie over a = a fibre of n entries, from the
// maxima of |a| over the unused entries of its DOT_SEG-entry segments (part[s * ldp + SEG_SLOT],
// written by the blocks of k_aca_post): the global maximum is the largest segment maximum, and
// the lowest index within the tie band lies in the first segment whose maximum reaches the
// band, so only that segment is scanned.
constexpr int SEG_SLOT = SLAR_MAX_RANK;   // slot of a partial-sum row left free by the dots (l < kmax)

__device__ void segment_argmax_tie(const double* a, int n, const unsigned char* used, const double* part, int ldp,
                                   int nseg, int* out_idx, double* out_max) {
  __shared__ double wmax[32];
  __shared__ int widx[32];
  __shared__ double top_s;
  __shared__ int seg_s;
  const int tid = threadIdx.x, nthr = blockDim.x, nw = blockDim.x >> 5;
  double m = -1.0;
  for (int q = tid; q < nseg; q += nthr) m = fmax(m, __ldcg(part + (long long)q * ldp + SEG_SLOT));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) wmax[tid >> 5] = m;
  __syncthreads();
  if (tid == 0) {
    double t = -1.0;
    for (int w = 0; w < nw; ++w) t = fmax(t, wmax[w]);
    top_s = t;
  }
  __syncthreads();
  const double top = top_s;
  const double thr = top * (1.0 - TIE_RTOL);
  int fs = 0x7fffffff;
  if (top >= 0.0)
    for (int q = tid; q < nseg; q += nthr)
      if (__ldcg(part + (long long)q * ldp + SEG_SLOT) >= thr && q < fs) fs = q;
  for (int o = 16; o > 0; o >>= 1) fs = min(fs, __shfl_down_sync(0xffffffffu, fs, o));
  if ((tid & 31) == 0) widx[tid >> 5] = fs;
  __syncthreads();
  if (tid == 0) {
    int b = 0x7fffffff;
    for (int w = 0; w < nw; ++w) b = min(b, widx[w]);
    seg_s = b;
  }
  __syncthreads();
  const int seg = seg_s;
  int best = 0x7fffffff;
  if (top >= 0.0 && seg != 0x7fffffff) {
    const long long thrk = __double_as_longlong(thr);
    const int end = min(n, (seg + 1) * DOT_SEG);
    for (int i = seg * DOT_SEG + tid; i < end; i += nthr)
      if (i < best && !used[i] && abs_key(a[i]) >= thrk) best = i;
  }
  for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_down_sync(0xffffffffu, best, o));
  __syncthreads();
  if ((tid & 31) == 0) widx[tid >> 5] = best;
  __syncthreads();
  if (tid == 0) {
    int b = 0x7fffffff;
    for (int w = 0; w < nw; ++w) b = min(b, widx[w]);
    *out_idx = (top >= 0.0 && b != 0x7fffffff) ? b : -1;
    *out_max = top;
  }
  __syncthreads();
}

__global__ void k_aca_init(AcaState* st, int* pivI, unsigned char* usedr, int replay, double eps, int cap_binds) {
  if (threadIdx.x != 0) return;
  st->k = 0;
  st->done = 0;
  st->stop_row = 0;
  st->replay = replay;
  st->eps = eps;
  st->tc_err = 0;
  st->normA2 = 0.0;
  st->cap_binds = cap_binds;
  st->capped = 0;
  st->piv0 = 0.0;
  st->skip = 0;
  st->n_skip = 0;
  if (!replay) pivI[0] = 0;
  if (pivI[0] < 0) { st->done = 1; return; }
  usedr[pivI[0]] = 1;
}

// column pivot from the residual row r, v_k = r / r[j_k].  A negligible row (largest unused
// entry <= max(NOISE_RTOL, eps / 100) |first pivot|) takes no pivot: like a vanishing term it goes to
// the check rows, which stop the approximation or name the next row (the unused check row of
// largest residual, written to pivI[k]); st->skip then makes this step's column fibre and
// post kernel return at once, and the next step samples that row.
__global__ void __launch_bounds__(PIV_THREADS)
k_aca_row_pivot(const double* __restrict__ r, int M1, int M2, unsigned char* usedc, unsigned char* usedr,
                int* pivI, int* pivJ, AcaState* st, double* __restrict__ Va, int n_chk,
                const int* __restrict__ chk_rows, const double* __restrict__ chk_n2) {
  __shared__ int j_s;
  __shared__ double top_s;
  if (st->done) return;
  const int kk = st->k;
  const int replay = st->replay;
  double* vout = Va + (long long)kk * M2;
  if (threadIdx.x == 0) st->skip = 0;   // the previous step's post kernel has finished with it
  if (replay) {
    if (threadIdx.x == 0) { j_s = pivJ[kk]; top_s = 1.0; }
    __syncthreads();
  } else {
    block_argmax_tie(r, M2, usedc, &j_s, &top_s);
    if (kk > 0 && top_s >= 0.0 && top_s <= fmax(NOISE_RTOL, 0.01 * st->eps) * st->piv0) {
      if (threadIdx.x == 0) {
        st->skip = 1;
        st->n_skip += 1;
        double n2c[8];
        double sum = 0.0;
        for (int q = 0; q < n_chk; ++q) {
          n2c[q] = chk_n2[q];
          sum += n2c[q];
        }
        int best = -1;
        if (n_chk > 0 && (double)M1 / n_chk * sum > st->eps * st->eps * st->normA2)
          for (int q = 0; q < n_chk; ++q)
            if (!usedr[chk_rows[q]] && (best < 0 || n2c[q] > n2c[best])) best = q;
        if (best < 0) {
          st->done = 1;       // confirmed (or no check row left): stop (the row is counted in n_skip)
        } else {
          pivI[kk] = chk_rows[best];
          usedr[chk_rows[best]] = 1;
        }
      }
      return;
    }
  }
  const int j = j_s;
  if (j < 0 || top_s == 0.0 || r[j] == 0.0) {
    if (threadIdx.x == 0) { st->done = 1; st->stop_row = replay ? 0 : 1; }
    return;
  }
  const double piv = r[j];
  // one reciprocal for the CTA instead of M2 FP64 divisions (a division costs about eight
  // FP64-pipe instructions, and every warp computing it serialises on the SM's few FP64
  // units); v_k[j] = 1 exactly
  __shared__ double inv_s;
  if (threadIdx.x == 0) inv_s = 1.0 / piv;
  __syncthreads();
  const double inv = inv_s;
  for (int i = threadIdx.x; i < M2; i += PIV_THREADS) vout[i] = i == j ? 1.0 : r[i] * inv;
  if (threadIdx.x == 0) {
    pivJ[kk] = j;
    usedc[j] = 1;
    st->piv = piv;
    if (kk == 0) st->piv0 = fabs(piv);
  }
  (void)M1;
  (void)pivI;
}

// norm estimate, stop test (confirmed on the check rows), next row pivot; run by the last
// block of k_aca_post (partial sums and check-row norms are read through L2)
__device__ void aca_finalize_body(const double* __restrict__ Ua, int M1, int kmax, int nbu, int nbv,
               const double* __restrict__ part, int ldp, AcaState* st, int* pivI,
               unsigned char* usedr, int n_chk, const int* __restrict__ chk_rows,
               const double* __restrict__ chk_n2, cudaGraphConditionalHandle loop, int use_cond) {
  __shared__ double du[SLAR_MAX_RANK + 1], dv[SLAR_MAX_RANK + 1];
  __shared__ int i_s;
  __shared__ double top_s;
  __shared__ int stop_s;
  __shared__ int next_s;
  const int tid = threadIdx.x;
  const int kk = st->k;
  const int replay = st->replay;
  const double eps = st->eps;
  __syncthreads();
  // the partials of dot l summed by one warp (lanes over blocks, shuffle tree): no thread
  // walks a chain of dependent L2 loads
  {
    const int warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
    for (int l = warp; l <= kk; l += nw) {
      double a = 0.0, b = 0.0;
      for (int blk = lane; blk < nbu; blk += 32) a += __ldcg(part + (long long)blk * ldp + l);
      for (int blk = nbu + lane; blk < nbu + nbv; blk += 32) b += __ldcg(part + (long long)blk * ldp + l);
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
      }
      if (lane == 0) {
        du[l] = a;
        dv[l] = b;
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    double cross = 0.0;
    for (int l = 0; l < kk; ++l) cross += du[l] * dv[l];
    const double nu2 = du[kk], nv2 = dv[kk];
    const double n2 = st->normA2 + 2.0 * cross + nu2 * nv2;
    st->normA2 = n2;
    st->k = kk + 1;
    int stop = 0;
    int next = -1;
    if (kk + 1 >= kmax) {
      stop = 1;
      // the cap ends the approximation although the rank-1 test is not met: eps is not
      // reached within the cap (a warning; the result is still a valid approximation)
      if (!replay && st->cap_binds && sqrt(nu2) * sqrt(nv2) > eps * sqrt(fmax(n2, 0.0))) st->capped = 1;
    } else if (!replay && sqrt(nu2) * sqrt(nv2) <= eps * sqrt(fmax(n2, 0.0))) {
      stop = 1;
      if (n_chk > 0) {
        double sum = 0.0;
        double n2c[8];
        for (int q = 0; q < n_chk; ++q) {
          n2c[q] = __ldcg(chk_n2 + q);
          sum += n2c[q];
        }
        if ((double)M1 / n_chk * sum > eps * eps * n2) {
          // the residual elsewhere is too large: continue from the worst unused check row
          int best = -1;
          for (int q = 0; q < n_chk; ++q)
            if (!usedr[chk_rows[q]] && (best < 0 || n2c[q] > n2c[best])) best = q;
          if (best >= 0) {
            stop = 0;
            next = chk_rows[best];
          }
        }
      }
    } else if (replay && pivI[kk + 1] < 0) {
      stop = 1;
    }
    if (stop) st->done = 1;
    stop_s = stop;
    next_s = next;
  }
  __syncthreads();
  if (!stop_s && next_s >= 0) {
    if (tid == 0) {
      pivI[kk + 1] = next_s;
      usedr[next_s] = 1;
      if (use_cond) cudaGraphSetConditional(loop, 1);
    }
    return;
  }
  if (stop_s) {
    if (tid == 0) if (use_cond) cudaGraphSetConditional(loop, 0);
    return;
  }
  if (replay) {
    if (tid == 0) {
      usedr[pivI[kk + 1]] = 1;
      if (use_cond) cudaGraphSetConditional(loop, 1);
    }
    return;
  }
  segment_argmax_tie(Ua + (long long)kk * M1, M1, usedr, part, ldp, nbu, &i_s, &top_s);
  if (tid == 0) {
    if (i_s < 0) {
      st->done = 1;
      if (use_cond) cudaGraphSetConditional(loop, 0);
    } else {
      pivI[kk + 1] = i_s;
      usedr[i_s] = 1;
      if (use_cond) cudaGraphSetConditional(loop, 1);
    }
  }
}

// One kernel after the column fibre: blocks [0, nbu + nbv) form the partial dot products of
// u_k with U_l and of v_k with V_l (l <= k), blocks [nbu + nbv, + n_chk) update the check-row
// residuals; the last block to finish (atomic ticket after a fence) runs the finalize step.
__global__ void __launch_bounds__(256)
k_aca_post(const double* __restrict__ Ua, int M1, const double* __restrict__ Va, int M2, int kmax, int nbu,
           int nbv, double* __restrict__ part, int ldp, AcaState* st, int* pivI, unsigned char* usedr, int n_chk,
           const int* __restrict__ chk_rows, double* __restrict__ chk_R, double* __restrict__ chk_n2,
           cudaGraphConditionalHandle loop, int use_cond) {
  __shared__ double red[8];
  __shared__ int s_last;
  if (st->done) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && use_cond) cudaGraphSetConditional(loop, 0);
    return;
  }
  if (st->skip) {   // a negligible row: no term this step, the next step samples pivI[k]
    if (blockIdx.x == 0 && threadIdx.x == 0 && use_cond) cudaGraphSetConditional(loop, 1);
    return;
  }
  const int kk = st->k;
  const int blk = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (blk < nbu + nbv) {
    const bool isu = blk < nbu;
    const double* X = isu ? Ua : Va;
    const int M = isu ? M1 : M2;
    const int s0 = (isu ? blk : blk - nbu) * DOT_SEG;
    const double* xk = X + (long long)kk * M;
    // the new factor's segment in registers; each warp takes two columns l per pass (16 loads
    // in flight per lane)
    constexpr int J = DOT_SEG / 32;
    double xr[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int i = s0 + lane + 32 * j;
      xr[j] = i < M ? xk[i] : 0.0;
    }
    for (int l = warp; l <= kk; l += 16) {   // columns l and l + 8
      const int l2 = l + 8;
      const bool has2 = l2 <= kk;
      double a = 0.0, b = 0.0;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int i = s0 + lane + 32 * j;
        a += (i < M ? X[(long long)l * M + i] : 0.0) * xr[j];
        b += ((has2 && i < M) ? X[(long long)l2 * M + i] : 0.0) * xr[j];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
      }
      if (lane == 0) {
        part[(long long)blk * ldp + l] = a;
        if (has2) part[(long long)blk * ldp + l2] = b;
      }
    }
    if (isu) {
      // maximum of |u_k| over the unused rows of this segment, for the next row pivot
      const int i = s0 + (int)threadIdx.x;   // DOT_SEG entries, one per thread
      long long m = (i < M && !usedr[i]) ? abs_key(xk[i]) : -1LL;
      m = warp_max_ll(m);
      if (lane == 0) red[warp] = __longlong_as_double(m);   // bit copy (-1 maps to a NaN pattern)
      __syncthreads();
      if (threadIdx.x == 0) {
        long long t = -1;
        for (int w = 0; w < 8; ++w) {
          const long long u = __double_as_longlong(red[w]);
          t = u > t ? u : t;
        }
        part[(long long)blk * ldp + SEG_SLOT] = t >= 0 ? __longlong_as_double(t) : -1.0;
      }
    }
  } else if (!st->replay) {
    const int c = blk - nbu - nbv;
    const double a = Ua[(long long)kk * M1 + chk_rows[c]];
    const double* v = Va + (long long)kk * M2;
    double* r = chk_R + (long long)c * M2;
    double sq = 0.0;
    for (int e = threadIdx.x; e < M2; e += 256) {
      const double t = r[e] - a * v[e];
      r[e] = t;
      sq += t * t;
    }
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
    if (lane == 0) red[warp] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[w];
      chk_n2[c] = t;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&st->post_ctr, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x == 0) st->post_ctr = 0;
  aca_finalize_body(Ua, M1, kmax, nbu, nbv, part, ldp, st, pivI, usedr, n_chk, chk_rows, chk_n2, loop, use_cond);
}


// ---------------------------------------------------------------------------------------
// Block cross approximation (slar_config.aca_block = b > 1): a step samples the residuals of
// the b rows pivI[k .. k + nrows) at once (rowbuf, b x M2), takes pivots in them in order --
// row t: arg-max j_t of its residual, v_t = r / r[j_t], and the later rows of the block lose
// r[t'][j_t] v_t -- samples the accepted columns at once (Ua columns k .., the residual
// against the previous k terms), turns them into the new column factors by forward
// substitution u_t = C_t - sum_{s<t} u_s v_s[j_t], and accepts the terms in order with the
// stop test of the one-fibre steps.  Negligible rows (as there) add no term.

// The next rows: up to nsel rows of largest |u| over the unused rows, each pick the lowest
// index within the tie band of the remaining maximum (block_argmax_tie); the picks are marked
// used (they are the next block's rows).  Called by every thread of the CTA.
__device__ void pick_rows(const double* u, int M1, unsigned char* usedr, int nsel, int* out, int* nout) {
  __shared__ int i_s;
  __shared__ double t_s;
  int n = 0;
  for (int p = 0; p < nsel; ++p) {
    block_argmax_tie(u, M1, usedr, &i_s, &t_s);
    const int i = i_s;
    if (i < 0) break;
    if (threadIdx.x == 0) {
      out[n] = i;
      usedr[i] = 1;
    }
    ++n;
    __syncthreads();
  }
  if (threadIdx.x == 0) *nout = n;
  __syncthreads();
}

// The check rows decide after a vanishing term or a passed rank-1 test: returns 1 (stop) or
// 0 with *redirect = the unused check row of largest residual norm n2c[q * stride].
__device__ __forceinline__ int check_decision(int M1, int n_chk, const int* chk_rows, const double* n2c, int stride,
                                              const unsigned char* usedr, double eps, double normA2, int* redirect) {
  double sum = 0.0;
  for (int q = 0; q < n_chk; ++q) sum += n2c[q * stride];
  if (n_chk == 0 || (double)M1 / n_chk * sum <= eps * eps * normA2) return 1;
  int best = -1;
  for (int q = 0; q < n_chk; ++q)
    if (!usedr[chk_rows[q]] && (best < 0 || n2c[q * stride] > n2c[best * stride])) best = q;
  if (best < 0) return 1;
  *redirect = chk_rows[best];
  return 0;
}

// the first block: row 0 and the first b - 1 check rows other than 0
__global__ void k_aca_block_init(AcaState* st, int* pivI, const int* chk_rows, int n_chk, int b, int kmax) {
  if (threadIdx.x != 0) return;
  int n = 0;
  pivI[n++] = 0;
  for (int q = 0; q < n_chk && n < b; ++q)
    if (chk_rows[q] != 0) pivI[n++] = chk_rows[q];
  st->nrows = n < kmax ? n : kmax;
  st->nact = 0;
  st->rows_sampled = 0;
  st->cols_sampled = 0;
  st->nsteps = 0;
}

// Pivots in the block's rows (one CTA).  rowbuf holds the rows' residuals against the k
// previous terms; they are reduced in place by the block's terms.
__global__ void __launch_bounds__(PIV_THREADS)
k_aca_block_pivot(double* __restrict__ rowbuf, int M1, int M2, unsigned char* usedc, unsigned char* usedr, int* pivI,
                  int* pivJ, AcaState* st, double* __restrict__ Va, const double* __restrict__ Ua, int n_chk,
                  const int* __restrict__ chk_rows, const double* __restrict__ chk_n2, int b, int kmax) {
  __shared__ int rows_s[ACA_BMAX], acc_s[ACA_BMAX];
  __shared__ double coef_s[ACA_BMAX];
  __shared__ int j_s, nacc_s, next_s[ACA_BMAX], nnext_s;
  __shared__ double top_s, piv0_s;
  if (st->done) return;
  const int tid = threadIdx.x;
  const int kk = st->k;
  const int nrows = st->nrows;
  if (tid == 0) {
    st->skip = 0;
    st->rows_sampled += nrows;
    st->nsteps += 1;
    nacc_s = 0;
    piv0_s = st->piv0;
  }
  if (tid < nrows) rows_s[tid] = pivI[kk + tid];
  __syncthreads();
  const double floor_rel = fmax(NOISE_RTOL, 0.01 * st->eps);
  for (int t = 0; t < nrows; ++t) {
    const double* r = rowbuf + (long long)t * M2;
    if (tid == 0) usedr[rows_s[t]] = 1;
    block_argmax_tie(r, M2, usedc, &j_s, &top_s);
    const double top = top_s, piv0 = piv0_s;
    if (piv0 == 0.0 && !(top > 0.0)) {
      // the first row of the call vanishes: nothing to approximate (the row was sampled)
      if (tid == 0) { st->done = 1; st->stop_row = 1; st->nact = 0; }
      return;
    }
    if (j_s < 0 || (piv0 > 0.0 && top <= floor_rel * piv0)) {   // negligible: no term
      if (tid == 0) st->n_skip += 1;
      __syncthreads();
      continue;
    }
    const int j = j_s;
    const double piv = r[j];
    const int a = nacc_s;
    double* vout = Va + (long long)(kk + a) * M2;
    __shared__ double inv_s;   // one FP64 division for the CTA
    if (tid == 0) inv_s = 1.0 / piv;
    __syncthreads();
    const double inv = inv_s;
    for (int i = tid; i < M2; i += PIV_THREADS) vout[i] = i == j ? 1.0 : r[i] * inv;
    if (tid < nrows) coef_s[tid] = tid > t ? rowbuf[(long long)tid * M2 + j] : 0.0;
    __syncthreads();
    if (tid == 0) {
      usedc[j] = 1;
      pivJ[kk + a] = j;
      acc_s[a] = rows_s[t];
      nacc_s = a + 1;
      if (piv0 == 0.0) {
        piv0_s = fabs(piv);
        st->piv0 = fabs(piv);
      }
    }
    for (int t2 = t + 1; t2 < nrows; ++t2) {
      const double cf = coef_s[t2];
      double* r2 = rowbuf + (long long)t2 * M2;
      for (int i = tid; i < M2; i += PIV_THREADS) r2[i] -= cf * vout[i];
    }
    __syncthreads();
  }
  const int nacc = nacc_s;
  if (tid < nacc) pivI[kk + tid] = acc_s[tid];
  if (tid == 0) {
    st->nact = nacc;
    st->cols_sampled += nacc;
  }
  if (nacc > 0) return;
  // every row of the block was negligible: a vanishing term for the stop test
  __shared__ int stop_s, redirect_s;
  if (tid == 0) {
    int redirect = -1;
    stop_s = check_decision(M1, n_chk, chk_rows, chk_n2, 1, usedr, st->eps, st->normA2, &redirect);
    redirect_s = redirect;
    st->skip = 1;
    if (stop_s) st->done = 1;
    else usedr[redirect] = 1;
  }
  __syncthreads();
  if (stop_s) return;
  // the next block: the check row, then the rows of largest |u| of the latest column
  const int room = kmax - kk;
  const int nsel = (b < room ? b : room) - 1;
  pick_rows(Ua + (long long)(kk - 1) * M1, M1, usedr, nsel, next_s, &nnext_s);
  if (tid == 0) {
    pivI[kk] = redirect_s;
    for (int q = 0; q < nnext_s; ++q) pivI[kk + 1 + q] = next_s[q];
    st->nrows = 1 + nnext_s;
  }
}

// forward substitution of the sampled columns: u_t = C_t - sum_{s<t} u_s v_s[j_t]
__global__ void k_aca_block_fsub(double* __restrict__ Ua, int M1, const double* __restrict__ Va, int M2,
                                 const int* __restrict__ pivJ, const AcaState* st) {
  __shared__ double vj[ACA_BMAX][ACA_BMAX];
  if (st->done || st->skip) return;
  const int kk = st->k, n = st->nact;
  if (n <= 1) return;
  if (threadIdx.x < n * n) {
    const int s = threadIdx.x / n, t = threadIdx.x - s * n;
    vj[s][t] = s < t ? Va[(long long)(kk + s) * M2 + pivJ[kk + t]] : 0.0;
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M1) return;
  double u[ACA_BMAX];
  for (int t = 0; t < n; ++t) {
    double x = Ua[(long long)(kk + t) * M1 + i];
    for (int s = 0; s < t; ++s) x -= u[s] * vj[s][t];
    u[t] = x;
    Ua[(long long)(kk + t) * M1 + i] = x;
  }
}

// After the columns: blocks [0, nbu) form the partial dots of the new u_t with every column
// of U (t < nact, l < k + nact), blocks [nbu, nbu + nbv) those of the new v_t with V, blocks
// [nbu + nbv, + n_chk) apply the new terms to the check rows and keep their norms after each
// term; the last block accepts the terms in order (norm estimate, rank-1 test, check rows),
// and picks the next block's rows.  A dot block keeps two new factors' segment in registers
// and each warp takes two columns l per pass (32 loads in flight per lane); the last block
// sums each dot's partials in one thread with four accumulators (fixed order) -- the dots
// are chains of L2 loads, and these are the loads that can be in flight at once.
__global__ void __launch_bounds__(256)
k_aca_block_post(const double* __restrict__ Ua, int M1, const double* __restrict__ Va, int M2, int kmax, int nbu,
                 int nbv, double* __restrict__ part, int ldp, AcaState* st, int* pivI, unsigned char* usedr, int n_chk,
                 const int* __restrict__ chk_rows, double* __restrict__ chk_R, double* __restrict__ chk_n2,
                 double* __restrict__ chk_n2t, int b, cudaGraphConditionalHandle loop, int use_cond) {
  __shared__ double red[8];
  __shared__ int s_last;
  if (st->done) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && use_cond) cudaGraphSetConditional(loop, 0);
    return;
  }
  if (st->skip) {   // every row of the block was negligible: the next block is set
    if (blockIdx.x == 0 && threadIdx.x == 0 && use_cond) cudaGraphSetConditional(loop, 1);
    return;
  }
  const int kk = st->k, na = st->nact, K = kk + na;
  const int blk = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (blk < nbu + nbv) {
    const bool isu = blk < nbu;
    const double* X = isu ? Ua : Va;
    const int M = isu ? M1 : M2;
    const int s0 = (isu ? blk : blk - nbu) * DOT_SEG;
    constexpr int J = DOT_SEG / 32;
    double* pb = part + (long long)blk * ldp;
    for (int t0 = 0; t0 < na; t0 += 2) {
      const bool two = t0 + 1 < na;
      double x0[J], x1[J];
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int i = s0 + lane + 32 * j;
        x0[j] = i < M ? X[(long long)(kk + t0) * M + i] : 0.0;
        x1[j] = (two && i < M) ? X[(long long)(kk + t0 + 1) * M + i] : 0.0;
      }
      for (int l = warp; l < K; l += 16) {   // columns l and l + 8
        const int l2 = l + 8;
        const bool has2 = l2 < K;
        double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int i = s0 + lane + 32 * j;
          const double y = i < M ? X[(long long)l * M + i] : 0.0;
          const double y2 = (has2 && i < M) ? X[(long long)l2 * M + i] : 0.0;
          a0 += y * x0[j];
          a1 += y * x1[j];
          b0 += y2 * x0[j];
          b1 += y2 * x1[j];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          a0 += __shfl_down_sync(0xffffffffu, a0, o);
          a1 += __shfl_down_sync(0xffffffffu, a1, o);
          b0 += __shfl_down_sync(0xffffffffu, b0, o);
          b1 += __shfl_down_sync(0xffffffffu, b1, o);
        }
        if (lane == 0) {
          pb[t0 * K + l] = a0;
          if (two) pb[(t0 + 1) * K + l] = a1;
          if (has2) {
            pb[t0 * K + l2] = b0;
            if (two) pb[(t0 + 1) * K + l2] = b1;
          }
        }
      }
    }
  } else {
    const int q = blk - nbu - nbv;
    double* r = chk_R + (long long)q * M2;
    for (int t = 0; t < na; ++t) {
      const double a = Ua[(long long)(kk + t) * M1 + chk_rows[q]];
      const double* v = Va + (long long)(kk + t) * M2;
      double sq = 0.0;
      for (int e = threadIdx.x; e < M2; e += 256) {
        const double x = r[e] - a * v[e];
        r[e] = x;
        sq += x * x;
      }
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
      if (lane == 0) red[warp] = sq;
      __syncthreads();
      if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        chk_n2t[q * ACA_BMAX + t] = s;
      }
      __syncthreads();
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&st->post_ctr, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // ---- finalize (last block) ----
  __shared__ double du[ACA_BMAX * (SLAR_MAX_RANK + ACA_BMAX)], dv[ACA_BMAX * (SLAR_MAX_RANK + ACA_BMAX)];
  __shared__ int stop_s, redirect_s, kend_s, next_s[ACA_BMAX], nnext_s;
  const int tid = threadIdx.x;
  if (tid == 0) st->post_ctr = 0;
  // the partials of dot w summed by one thread (four accumulators, fixed order)
  auto sum4 = [&](const double* p0, int nb, int w) {   // partials nb apart by ldp, four chains
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int q = 0;
    for (; q + 4 <= nb; q += 4) {
      a0 += __ldcg(p0 + (long long)q * ldp + w);
      a1 += __ldcg(p0 + (long long)(q + 1) * ldp + w);
      a2 += __ldcg(p0 + (long long)(q + 2) * ldp + w);
      a3 += __ldcg(p0 + (long long)(q + 3) * ldp + w);
    }
    for (; q < nb; ++q) a0 += __ldcg(p0 + (long long)q * ldp + w);
    return (a0 + a1) + (a2 + a3);
  };
  for (int w = tid; w < na * K; w += 256) {
    du[w] = sum4(part, nbu, w);
    dv[w] = sum4(part + (long long)nbu * ldp, nbv, w);
  }
  __syncthreads();
  if (tid == 0) {
    double n2 = st->normA2;
    const double eps = st->eps;
    int stop = 0, redirect = -1, kend = K;
    for (int t = 0; t < na; ++t) {
      double cross = 0.0;
      for (int l = 0; l < kk + t; ++l) cross += du[t * K + l] * dv[t * K + l];
      const double nu2 = du[t * K + kk + t], nv2 = dv[t * K + kk + t];
      n2 = n2 + 2.0 * cross + nu2 * nv2;
      const bool small = sqrt(nu2) * sqrt(nv2) <= eps * sqrt(fmax(n2, 0.0));
      if (kk + t + 1 >= kmax) {
        stop = 1;
        kend = kk + t + 1;
        if (st->cap_binds && !small) st->capped = 1;
        break;
      }
      if (small) {
        int rd = -1;
        if (check_decision(M1, n_chk, chk_rows, chk_n2t + t, ACA_BMAX, usedr, eps, n2, &rd)) {
          stop = 1;
          kend = kk + t + 1;
          break;
        }
        redirect = rd;
      }
    }
    st->normA2 = n2;
    st->k = kend;
    const int tl = kend - kk - 1;
    for (int q = 0; q < n_chk; ++q) chk_n2[q] = chk_n2t[q * ACA_BMAX + tl];
    if (stop) st->done = 1;
    else if (redirect >= 0) usedr[redirect] = 1;
    stop_s = stop;
    redirect_s = redirect;
    kend_s = kend;
  }
  __syncthreads();
  if (stop_s) {
    if (tid == 0 && use_cond) cudaGraphSetConditional(loop, 0);
    return;
  }
  const int kend = kend_s;
  const int room = kmax - kend;
  const int nsel = (b < room ? b : room) - (redirect_s >= 0 ? 1 : 0);
  pick_rows(Ua + (long long)(kend - 1) * M1, M1, usedr, nsel, next_s, &nnext_s);
  if (tid == 0) {
    int n = 0;
    if (redirect_s >= 0) pivI[kend + n++] = redirect_s;
    for (int q = 0; q < nnext_s; ++q) pivI[kend + n++] = next_s[q];
    st->nrows = n;
    if (n == 0) st->done = 1;
    if (use_cond) cudaGraphSetConditional(loop, n > 0 ? 1 : 0);
  }
}
}  // namespace

// One cross-approximation step: row fibre with residual, column pivot and v_k, column
// fibre into u_k, dot products, norm estimate / stop test / next row pivot.  All kernels
// read the step index from the device state.  With `prof` the two evaluator launches are
// bracketed by CUDA events.
slar_status aca_step(slar_ctx* c, size_t smem, cudaGraphConditionalHandle h, int use_cond, bool prof) {
  cudaStream_t s = c->s;
  const int M1 = c->M1, M2 = c->M2;
  const int nbu = (M1 + DOT_SEG - 1) / DOT_SEG, nbv = (M2 + DOT_SEG - 1) / DOT_SEG;
  const int ldp = SLAR_MAX_RANK + 1;
  EvalArgs ar{};
  ar.mode = EVAL_ROW;
  ar.n = M2;
  ar.pivot = c->pivI;
  ar.kidx = &c->ast->k;
  ar.out_stride = 0;
  ar.done = &c->ast->done;
  ar.X = c->Ua;
  ar.ldX = M1;
  ar.Y = c->Va;
  ar.ldY = M2;
  ar.out = c->rowbuf;
  EvalArgs ac = ar;
  ac.mode = EVAL_COL;
  ac.n = M1;
  ac.pivot = c->pivJ;
  ac.X = c->Va;
  ac.ldX = M2;
  ac.Y = c->Ua;
  ac.ldY = M1;
  ac.out = c->Ua;
  ac.out_stride = M1;
  ac.skip = &c->ast->skip;   // no column fibre after a negligible row
  const bool f32 = c->cfg.precision != SLAR_FP64;
  const int tc = tc_pieces(c);
  for (int pass = 0; pass < 2; ++pass) {
    const EvalArgs& a = pass == 0 ? ar : ac;
    const bool ev = prof && c->prof_n * 2 + 1 < kProfEvents;
    if (ev) CK(cudaEventRecord(c->prof_ev[2 * c->prof_n], s));
    cudaError_t e =
        tc ? launch_sl_eval_tc_dev(c->g, static_cast<const EvalParams<float>*>(c->evp), a, c->tc_b12, c->tc_b34,
                                   c->tc_broot, &c->ast->tc_err, tc, smem, c->tc_sc, s)
        : f32 ? launch_sl_eval_dev<float>(c->g, static_cast<const EvalParams<float>*>(c->evp), a, smem, s,
                                          c->eval_tile)
              : launch_sl_eval_dev<double>(c->g, static_cast<const EvalParams<double>*>(c->evp), a, smem, s,
                                           c->eval_tile);
    CK(e);
    if (ev) {
      CK(cudaEventRecord(c->prof_ev[2 * c->prof_n + 1], s));
      c->prof_n++;
    }
    if (pass == 0)
      slar::count_launch(), k_aca_row_pivot<<<1, PIV_THREADS, 0, s>>>(c->rowbuf, M1, M2, c->usedc, c->usedr,
                                                                       c->pivI, c->pivJ, c->ast, c->Va, c->n_chk,
                                                                       c->chk_rows, c->chk_n2);
  }
  slar::count_launch(), k_aca_post<<<nbu + nbv + c->n_chk, 256, 0, s>>>(
      c->Ua, M1, c->Va, M2, c->kmax, nbu, nbv, c->aca_part, ldp, c->ast, c->pivI, c->usedr, c->n_chk, c->chk_rows,
      c->chk_R, c->chk_n2, h, use_cond);
  CK(cudaGetLastError());
  return SLAR_OK;
}

// One block cross-approximation step: the block's row fibres (residual against the k
// previous terms), the pivots in them, the accepted column fibres, forward substitution,
// and the post kernel (dots, check rows, stop test, next rows).  Reads k, the rows and the
// counts from the device state.
slar_status aca_block_step(slar_ctx* c, size_t smem, cudaGraphConditionalHandle h, int use_cond, bool prof) {
  cudaStream_t s = c->s;
  const int M1 = c->M1, M2 = c->M2;
  const int b = c->cfg.aca_block;
  const int nbu = (M1 + DOT_SEG - 1) / DOT_SEG, nbv = (M2 + DOT_SEG - 1) / DOT_SEG;
  const int ldp = ACA_BMAX * (SLAR_MAX_RANK + ACA_BMAX) + 1;
  EvalArgs ar{};
  ar.mode = EVAL_ROW;
  ar.n = (long long)b * M2;
  ar.nper = M2;
  ar.nact = &c->ast->nrows;
  ar.pivot = c->pivI;
  ar.kidx = &c->ast->k;
  ar.out_stride = 0;
  ar.done = &c->ast->done;
  ar.X = c->Ua;
  ar.ldX = M1;
  ar.Y = c->Va;
  ar.ldY = M2;
  ar.out = c->rowbuf;
  EvalArgs ac = ar;
  ac.mode = EVAL_COL;
  ac.n = (long long)b * M1;
  ac.nper = M1;
  ac.nact = &c->ast->nact;
  ac.pivot = c->pivJ;
  ac.X = c->Va;
  ac.ldX = M2;
  ac.Y = c->Ua;
  ac.ldY = M1;
  ac.out = c->Ua;
  ac.out_stride = M1;
  ac.skip = &c->ast->skip;
  const bool f32 = c->cfg.precision != SLAR_FP64;
  const int tc = tc_pieces(c);
  for (int pass = 0; pass < 2; ++pass) {
    const EvalArgs& a = pass == 0 ? ar : ac;
    const bool ev = prof && c->prof_n * 2 + 1 < kProfEvents;
    if (ev) CK(cudaEventRecord(c->prof_ev[2 * c->prof_n], s));
    cudaError_t e =
        tc ? launch_sl_eval_tc_dev(c->g, static_cast<const EvalParams<float>*>(c->evp), a, c->tc_b12, c->tc_b34,
                                   c->tc_broot, &c->ast->tc_err, tc, smem, c->tc_sc, s)
        : f32 ? launch_sl_eval_dev<float>(c->g, static_cast<const EvalParams<float>*>(c->evp), a, smem, s,
                                          c->eval_tile)
              : launch_sl_eval_dev<double>(c->g, static_cast<const EvalParams<double>*>(c->evp), a, smem, s,
                                           c->eval_tile);
    CK(e);
    if (ev) {
      CK(cudaEventRecord(c->prof_ev[2 * c->prof_n + 1], s));
      c->prof_n++;
    }
    if (pass == 0)
      slar::count_launch(), k_aca_block_pivot<<<1, PIV_THREADS, 0, s>>>(
          c->rowbuf, M1, M2, c->usedc, c->usedr, c->pivI, c->pivJ, c->ast, c->Va, c->Ua, c->n_chk, c->chk_rows,
          c->chk_n2, b, c->kmax);
  }
  slar::count_launch(), k_aca_block_fsub<<<(M1 + 255) / 256, 256, 0, s>>>(c->Ua, M1, c->Va, M2, c->pivJ, c->ast);
  slar::count_launch(), k_aca_block_post<<<nbu + nbv + c->n_chk, 256, 0, s>>>(
      c->Ua, M1, c->Va, M2, c->kmax, nbu, nbv, c->aca_part, ldp, c->ast, c->pivI, c->usedr, c->n_chk, c->chk_rows,
      c->chk_R, c->chk_n2, c->chk_n2t, b, h, use_cond);
  CK(cudaGetLastError());
  return SLAR_OK;
}

// Capture one cross-approximation step (row fibre, column pivot, column fibre, dot products,
// stop test / next row pivot) as the body of a WHILE conditional node.  The body reads the
// step index from the device state and the evaluator parameters from c->evp.
slar_status build_aca_graph(slar_ctx* c, size_t smem, bool block) {
  CaptureScope scope(c);
  cudaStream_t s = c->s;
  cudaGraphExec_t& ge = block ? c->aca_graph_blk : c->aca_graph;
  if (ge) {
    CK(cudaGraphExecDestroy(ge));
    ge = nullptr;
  }
  const long long l0 = launch_count();
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
  // two pivot steps per loop iteration: the second one's kernels exit at once when the first
  // has stopped the approximation (device flag), and both report the stop to the WHILE node
  for (int u = 0; u < ACA_UNROLL; ++u) CKS(block ? aca_block_step(c, smem, h, 1, false) : aca_step(c, smem, h, 1, false));
  cudaGraph_t body_out;
  CK(cudaStreamEndCapture(s, &body_out));
  CK(cudaGraphInstantiate(&ge, gl, 0));
  CK(cudaGraphDestroy(gl));
  const long long l1 = launch_count();
  add_launches(-(l1 - l0));
  if (block) {
    c->aca_graph_blk_nodes = l1 - l0;
    c->aca_graph_blk_smem = smem;
    c->aca_graph_blk_tile = c->eval_tile;
  } else {
    c->aca_graph_nodes = l1 - l0;
    c->aca_graph_smem = smem;
    c->aca_graph_tile = c->eval_tile;
  }
  return SLAR_OK;
}

namespace {

// Autotuner of the entry evaluator's tile (entries per CTA): per (tree, precision, grid,
// rank bucket) the candidates 16, 32, 64 are timed on the check-row evaluation of the
// first SLAR call that meets the key (two launches each, CUDA events); the fastest is kept
// for the process.
using TuneKey = std::tuple<int, int, int, int, int, int, int>;
std::map<TuneKey, int> g_tile_cache;
std::mutex g_tile_mutex;

int rank_bucket(const int* r6, int d) {
  int mx = 1;
  for (int i = 0; i < (d == 4 ? 6 : 2); ++i) mx = std::max(mx, r6[i]);
  int b = 8;
  while (b < mx) b *= 2;
  return b;
}

TuneKey tune_key(const slar_ctx* c, const int* r6) {
  return TuneKey(c->d, c->cfg.precision, c->g.N[0], c->g.N[1], c->g.N[2], c->g.N[3], rank_bucket(r6, c->d));
}

}  // namespace

// Evaluate the check rows of a SLAR call into c->chk_R (and, the first time a tuning key is
// met, choose the evaluator tile on this work).
slar_status eval_check_rows(slar_ctx* c, int in, bool with_corr, double tau, const double* E) {
  EvalArgs a{};
  a.mode = EVAL_TUPLES;
  a.n = (long long)c->n_chk * c->M2;
  a.idx = c->chk_idx;
  a.out = c->chk_R;
  a.tau = tau;
  a.E = E;
  a.foot_euler = (c->cfg.flags & SLAR_FOOT_EULER) ? 1 : 0;
  if (tc_pieces(c) > 0) {
    c->eval_tile = 128;   // the tensor-core evaluator's fixed MMA tile
    return eval_entries(c, in, with_corr, a, 0);
  }
  if (c->cfg.flags & SLAR_NO_AUTOTUNE) {
    c->eval_tile = 32;
    return eval_entries(c, in, with_corr, a, 0);
  }
  const TuneKey key = tune_key(c, c->ht[in].r);
  int tile = 0;
  {
    std::lock_guard<std::mutex> lock(g_tile_mutex);
    auto it = g_tile_cache.find(key);
    if (it != g_tile_cache.end()) tile = it->second;
  }
  if (tile) {
    c->eval_tile = tile;
    return eval_entries(c, in, with_corr, a, 0);
  }
  const int cand[3] = {16, 32, 64};
  float best_ms = 1e30f;
  int best = 16;
  const bool f32 = c->cfg.precision != SLAR_FP64;
  for (int q = 0; q < 3; ++q) {
    // a tile whose shared memory does not fit at these ranks is not a candidate
    const int fit = f32 ? sl_eval_fit_tile<float>(c->g, c->ht[in].r, cand[q])
                        : sl_eval_fit_tile<double>(c->g, c->ht[in].r, cand[q]);
    if (fit != cand[q]) continue;
    c->eval_tile = cand[q];
    CKS(eval_entries(c, in, with_corr, a, 0));   // warm-up (and the values, if last)
    // the better of two rounds of two launches: one round is easily disturbed (a choice
    // made here stays for the process)
    float ms = 1e30f;
    for (int round = 0; round < 2; ++round) {
      CK(cudaEventRecord(c->tune_ev[0], c->s));
      CKS(eval_entries(c, in, with_corr, a, 0));
      CKS(eval_entries(c, in, with_corr, a, 0));
      CK(cudaEventRecord(c->tune_ev[1], c->s));
      CK(cudaEventSynchronize(c->tune_ev[1]));
      float r = 0.f;
      CK(cudaEventElapsedTime(&r, c->tune_ev[0], c->tune_ev[1]));
      ms = r < ms ? r : ms;
    }
    if (ms < best_ms) { best_ms = ms; best = cand[q]; }
  }
  c->eval_tile = best;
  {
    std::lock_guard<std::mutex> lock(g_tile_mutex);
    g_tile_cache[key] = best;
  }
  return eval_entries(c, in, with_corr, a, 0);
}

slar_status slar_call(slar_ctx* c, int in, bool with_corr, double tau, const double* E, int out,
                      int* aca_rank, long long* entries) {
  cudaStream_t s = c->s;
  const int M1 = c->M1, M2 = c->M2;
  const int kmax = c->kmax;
  if (in == out) return set_error(c, SLAR_EINVAL, "SLAR output slot equals input slot");
  const bool replay = c->replay_pos < c->replay_calls;
  phase(c, PH_ACA);
  CK(cudaMemsetAsync(c->usedr, 0, M1, s));
  CK(cudaMemsetAsync(c->usedc, 0, M2, s));
  if (replay) {
    std::vector<int> I(kmax, -1), J(kmax, -1);
    const int* src = c->replay.data() + (size_t)c->replay_pos * c->replay_kmax * 2;
    for (int k = 0; k < kmax && k < c->replay_kmax; ++k) {
      I[k] = src[2 * k];
      J[k] = src[2 * k + 1];
      if (I[k] < 0 || J[k] < 0) { I[k] = J[k] = -1; break; }
      if (I[k] >= M1 || J[k] >= M2)
        return set_error(c, SLAR_EINVAL, "replayed pivot outside the matricisation");
    }
    CK(cudaMemcpy(c->pivI, I.data(), sizeof(int) * kmax, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->pivJ, J.data(), sizeof(int) * kmax, cudaMemcpyHostToDevice));
    c->replay_pos++;
  }
  // per-call evaluator parameters in device memory, read by the captured graph
  const HTBuf& hin = c->ht[in];
  const bool f32 = c->cfg.precision != SLAR_FP64;
  const int tc = tc_pieces(c);
  if (f32) CKS(refresh_f32_slot(c, in));
  if (f32) CKS(refresh_f32_fields(c, E, with_corr));
  if (f32) {
    EvalParams<float>* P = static_cast<EvalParams<float>*>(c->evp_host);
    P->ht = view32_slot(c, in);
    P->corr = corr_view(c, with_corr);
    P->tau = tau;
    P->E = E;
    P->E32 = c->E32;
    P->foot_euler = (c->cfg.flags & SLAR_FOOT_EULER) ? 1 : 0;
  } else {
    EvalParams<double>* P = static_cast<EvalParams<double>*>(c->evp_host);
    P->ht = view64(c, in);
    P->corr = corr_view(c, with_corr);
    P->tau = tau;
    P->E = E;
    P->foot_euler = (c->cfg.flags & SLAR_FOOT_EULER) ? 1 : 0;
  }
  CK(cudaMemcpyAsync(c->evp, c->evp_host, sizeof(EvalParams<double>), cudaMemcpyHostToDevice, s));
  const bool block = !replay && c->cfg.aca_block > 1;
  slar::count_launch(), k_aca_init<<<1, 32, 0, s>>>(c->ast, c->pivI, c->usedr, replay ? 1 : 0, c->cfg.eps,
                                                    kmax < std::min(M1, M2) ? 1 : 0);
  CK(cudaGetLastError());
  if (block) {
    slar::count_launch(), k_aca_block_init<<<1, 32, 0, s>>>(c->ast, c->pivI, c->chk_rows, c->n_chk,
                                                            c->cfg.aca_block, kmax);
    CK(cudaGetLastError());
  }
  long long chk_entries = 0;
  if (!replay && c->n_chk > 0) {
    // residuals of the check rows start as the rows themselves (this also fixes the tile)
    CKS(eval_check_rows(c, in, with_corr, tau, E));
    chk_entries = (long long)c->n_chk * M2;
  }
  if (!tc)
    c->eval_tile = f32 ? sl_eval_fit_tile<float>(c->g, hin.r, c->eval_tile)
                       : sl_eval_fit_tile<double>(c->g, hin.r, c->eval_tile);
  const size_t need = tc ? sl_eval_tc_smem(hin.r, tc)
                         : f32 ? sl_eval_smem<float>(c->g, hin.r, c->eval_tile)
                               : sl_eval_smem<double>(c->g, hin.r, c->eval_tile);
  const bool prof = (c->cfg.flags & SLAR_PROFILE_EVAL) != 0;
  // a graph is rebuilt when a call needs more evaluator shared memory than it was built with;
  // ranks grow over a run, so the SIMT evaluator's graph takes a quarter more than the call
  // needs (up to the 200 KB limit), which spares most rebuilds
  const size_t build = tc ? need : std::max(need, std::min<size_t>(need + need / 4, 200 * 1024));
  if (!prof && !block && (!c->aca_graph || need > c->aca_graph_smem || c->aca_graph_tile != c->eval_tile))
    CKS(build_aca_graph(c, build, false));
  if (!prof && block &&
      (!c->aca_graph_blk || need > c->aca_graph_blk_smem || c->aca_graph_blk_tile != c->eval_tile))
    CKS(build_aca_graph(c, build, true));
  if (prof) {
    // individually launched steps with events around the evaluator (roofline timing)
    // bounded like the WHILE loop: each step adds a term (at most kmax) or consumes a check
    // row after a negligible row (at most n_chk), or stops
    for (int it = 0; it < kmax + c->n_chk + 1; ++it) {
      CK(cudaMemcpyAsync(c->ast_host, c->ast, sizeof(AcaState), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (c->ast_host->done) break;   // where the WHILE node would stop
      CKS(block ? aca_block_step(c, need, 0, 0, true) : aca_step(c, need, 0, 0, true));
    }
  } else {
    CK(cudaGraphLaunch(block ? c->aca_graph_blk : c->aca_graph, s));
  }
  CK(cudaMemcpyAsync(c->ast_host, c->ast, sizeof(AcaState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const int k = c->ast_host->k;
  if (c->ast_host->capped) c->rank_capped++;
  if (c->ast_host->tc_err)
    return set_error(c, SLAR_ETIMEOUT, "tensor-core evaluator: an MMA completion wait ran out");
  long long nent;
  if (block) {
    // every sampled fibre counts, including the rows and columns of terms a stop dropped
    const int rows = c->ast_host->rows_sampled, cols = c->ast_host->cols_sampled;
    if (!prof)
      add_launches(c->aca_graph_blk_nodes * (long long)((c->ast_host->nsteps + ACA_UNROLL - 1) / ACA_UNROLL));
    nent = (long long)rows * M2 + (long long)cols * M1 + chk_entries;
  } else {
    // rows sampled without a term: negligible rows, and a vanishing first row
    const int extra_rows = c->ast_host->n_skip + c->ast_host->stop_row;
    if (!prof)
      add_launches(c->aca_graph_nodes * (long long)((k + extra_rows + ACA_UNROLL - 1) / ACA_UNROLL));
    nent = (long long)k * (M1 + M2) + (long long)extra_rows * M2 + chk_entries;
  }
  if (aca_rank) *aca_rank = k;
  if (entries) *entries = nent;
  c->prof_flop += (double)nent * entry_flops(c, in);
  if (k == 0) return set_error(c, SLAR_ENAN, "cross approximation found no pivot (zero tensor)");
  // exact HT embedding of U V^T, then HSVD truncation
  phase(c, PH_TRUNC);
  TruncIn tin;
  tin.d = c->d;
  tin.fast_qr = true;
  if (c->d == 4) {
    for (int m = 0; m < 4; ++m) {
      tin.U[m] = nullptr;
      tin.r[m] = c->g.N[m];
    }
    tin.r[4] = tin.r[5] = k;
    tin.B12 = c->Ua;
    tin.B34 = c->Va;
  } else {
    CK(transpose(c->Ua, k, M1, c->Lt[0], s));
    CK(transpose(c->Va, k, M2, c->Lt[1], s));
    tin.U[0] = c->Lt[0];
    tin.U[1] = c->Lt[1];
    tin.U[2] = tin.U[3] = nullptr;
    tin.r[0] = tin.r[1] = k;
    tin.r[2] = tin.r[3] = tin.r[4] = tin.r[5] = 0;
    tin.B12 = tin.B34 = nullptr;
  }
  CK(fill_identity(c->Ik, k, k, s));
  tin.Broot = c->Ik;
  return truncate_into(c, tin, c->cfg.eps, c->cfg.rank_cap, out);
}

}  // namespace slar
