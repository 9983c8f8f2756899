// Learned JFNK warm start: a four-layer periodic 3x3 convolutional network on the spatial
// grid (FP32) with its forward pass, backward pass, loss and Adam update as kernels.
//
// Layout: activations are [batch][channel][n0][n1] (row-major spatial grid, NX = n0 n1);
// parameters are one flat vector, per layer W[Cout][Cin][3][3] then bias[Cout].
//
// Kernels
//   k_conv<TW>      forward convolution (+ bias, + tanh) or its adjoint in the input (the
//                   convolution with transposed channels and flipped taps, times the tanh
//                   derivative 1 - h^2 of the layer below).  A CTA computes a TH x TW tile
//                   of output pixels (TH TW = 256, one pixel per thread) for all output
//                   channels; input halo tiles and weights are staged in shared memory in
//                   chunks of 8 input channels.
//   k_conv_wgrad<TW> per-(sample, tile) partial weight and bias gradients: each thread owns
//                   up to four (out, in) channel pairs and accumulates their nine taps over
//                   the tile's 256 pixels from shared memory; k_sum_cols reduces the
//                   partials over tiles and samples in a fixed order.
//   k_loss          loss terms and dL/dy per pixel with per-CTA partial sums.
//   k_adam          elementwise Adam update.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"

struct slar_net {
  int m = 0, hidden = 0, n0 = 0, n1 = 0, NX = 0, max_batch = 0;
  int cin[4] = {0, 0, 0, 0}, cout[4] = {0, 0, 0, 0};
  long long woff[4] = {0, 0, 0, 0}, boff[4] = {0, 0, 0, 0};
  long long np = 0;
  int TW = 16, TH = 16, tiles = 0;
  cudaStream_t s = nullptr;
  float* theta = nullptr;
  float* grad = nullptr;
  float* am = nullptr;
  float* av = nullptr;
  float* act[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  float* dA = nullptr;
  float* dB = nullptr;
  float* part = nullptr;
  long long part_len = 0;
  double* lpart = nullptr;
  double* loss_dev = nullptr;
  double* loss_host = nullptr;  // pinned
  long long t = 0;              // Adam steps taken
};

namespace slar {
namespace {

constexpr int CHUNK = 8;        // input channels staged per pass
constexpr int MAXC = 32;        // channel limit of every layer

__host__ __device__ constexpr int tile_h(int tw) { return 256 / tw; }
__host__ __device__ constexpr int halo_len(int tw) { return (tile_h(tw) + 2) * (tw + 2); }

// Forward (transpose = 0): out[o] = bias[o] + sum_{c,p,q} W[o][c][p][q] in[c][i+p-1][j+q-1],
// then tanh if act.  Adjoint (transpose = 1): out[c] = sum_{o,p,q} W[o][c][p][q]
// in[o][i-p+1][j-q+1], times (1 - gate[c]^2) if gate.  ci / co are the kernel's own input /
// output channel counts; ldw_in is the layer's Cin (row length of W).
template <int TW>
__global__ void __launch_bounds__(256) k_conv(const float* __restrict__ in, int ci,
                                              const float* __restrict__ W, const float* __restrict__ bias,
                                              float* __restrict__ out, int co, int n0, int n1, int transpose,
                                              int ldw_in, int act, const float* __restrict__ gate) {
  constexpr int TH = tile_h(TW);
  constexpr int HL = halo_len(TW);
  __shared__ float s_in[CHUNK][HL];
  __shared__ float s_w[MAXC][CHUNK][9];
  const int NX = n0 * n1;
  const int tiles1 = (n1 + TW - 1) / TW;
  const int ti0 = (blockIdx.x / tiles1) * TH, tj0 = (blockIdx.x % tiles1) * TW;
  const int b = blockIdx.y;
  const int li = threadIdx.x / TW, lj = threadIdx.x % TW;
  const int gi = ti0 + li, gj = tj0 + lj;
  const float* inb = in + (long long)b * ci * NX;
  float acc[MAXC];
#pragma unroll
  for (int o = 0; o < MAXC; ++o) acc[o] = 0.f;
  for (int c0 = 0; c0 < ci; c0 += CHUNK) {
    const int cn = min(CHUNK, ci - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < cn * HL; e += 256) {
      const int cc = e / HL, r = e % HL;
      const int hi = r / (TW + 2), hj = r % (TW + 2);
      int ii = (ti0 + hi - 1) % n0;
      if (ii < 0) ii += n0;
      int jj = (tj0 + hj - 1) % n1;
      if (jj < 0) jj += n1;
      s_in[cc][r] = inb[(long long)(c0 + cc) * NX + ii * n1 + jj];
    }
    for (int e = threadIdx.x; e < co * cn * 9; e += 256) {
      const int o = e / (cn * 9), r = e % (cn * 9);
      const int cc = r / 9, tap = r % 9;
      float wv;
      if (!transpose) wv = W[((long long)o * ldw_in + c0 + cc) * 9 + tap];
      else wv = W[((long long)(c0 + cc) * ldw_in + o) * 9 + (8 - tap)];
      s_w[o][cc][tap] = wv;
    }
    __syncthreads();
    for (int cc = 0; cc < cn; ++cc) {
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const float v = s_in[cc][(li + tap / 3) * (TW + 2) + lj + tap % 3];
#pragma unroll
        for (int o = 0; o < MAXC; ++o)
          if (o < co) acc[o] = fmaf(s_w[o][cc][tap], v, acc[o]);
      }
    }
  }
  if (gi >= n0 || gj >= n1) return;
  const long long px = (long long)gi * n1 + gj;
  float* ob = out + (long long)b * co * NX;
  const float* gb = gate ? gate + (long long)b * co * NX : nullptr;
#pragma unroll
  for (int o = 0; o < MAXC; ++o) {
    if (o >= co) break;
    float v = acc[o];
    if (bias) v += bias[o];
    if (act) v = tanhf(v);
    if (gb) {
      const float g = gb[(long long)o * NX + px];
      v *= 1.f - g * g;
    }
    ob[(long long)o * NX + px] = v;
  }
}

// Partial gradients of one layer for the tile blockIdx.x of sample blockIdx.y:
// part[cta][(o*ci + c)*9 + tap] = sum_px dz[o][px] x[c][px + off(tap)], then part[..][co*ci*9 + o]
// = sum_px dz[o][px].
template <int TW>
__global__ void __launch_bounds__(256) k_conv_wgrad(const float* __restrict__ x, int ci,
                                                    const float* __restrict__ dz, int co, int n0, int n1,
                                                    float* __restrict__ part, long long ldp) {
  constexpr int TH = tile_h(TW);
  constexpr int HL = halo_len(TW);
  constexpr int HLP = HL | 1;   // odd channel stride: conflict-free reads across channels
  extern __shared__ float smem[];
  float* s_x = smem;                  // [ci][HLP]
  float* s_d = smem + ci * HLP;       // [co][256]
  const int NX = n0 * n1;
  const int tiles1 = (n1 + TW - 1) / TW;
  const int ti0 = (blockIdx.x / tiles1) * TH, tj0 = (blockIdx.x % tiles1) * TW;
  const int b = blockIdx.y;
  const float* xb = x + (long long)b * ci * NX;
  const float* db = dz + (long long)b * co * NX;
  for (int e = threadIdx.x; e < ci * HL; e += 256) {
    const int c = e / HL, r = e % HL;
    const int hi = r / (TW + 2), hj = r % (TW + 2);
    int ii = (ti0 + hi - 1) % n0;
    if (ii < 0) ii += n0;
    int jj = (tj0 + hj - 1) % n1;
    if (jj < 0) jj += n1;
    s_x[c * HLP + r] = xb[(long long)c * NX + ii * n1 + jj];
  }
  for (int e = threadIdx.x; e < co * 256; e += 256) {
    const int o = e / 256, p = e % 256;
    const int gi = ti0 + p / TW, gj = tj0 + p % TW;
    s_d[o * 256 + p] = (gi < n0 && gj < n1) ? db[(long long)o * NX + gi * n1 + gj] : 0.f;
  }
  __syncthreads();
  const long long cta = (long long)blockIdx.y * gridDim.x + blockIdx.x;
  float* pp = part + cta * ldp;
  const int npair = co * ci;
  for (int pr0 = 0; pr0 < npair; pr0 += 1024) {
    float acc[4][9];
    int o_[4], c_[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int pr = pr0 + threadIdx.x + 256 * k;
      o_[k] = pr < npair ? pr / ci : -1;
      c_[k] = pr < npair ? pr % ci : 0;
#pragma unroll
      for (int t = 0; t < 9; ++t) acc[k][t] = 0.f;
    }
    for (int p = 0; p < 256; ++p) {
      const int li = p / TW, lj = p % TW;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (o_[k] < 0) continue;
        const float d = s_d[o_[k] * 256 + p];
        const float* xs = s_x + c_[k] * HLP + li * (TW + 2) + lj;
#pragma unroll
        for (int t = 0; t < 9; ++t) acc[k][t] = fmaf(d, xs[(t / 3) * (TW + 2) + t % 3], acc[k][t]);
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (o_[k] < 0) continue;
#pragma unroll
      for (int t = 0; t < 9; ++t) pp[((long long)o_[k] * ci + c_[k]) * 9 + t] = acc[k][t];
    }
  }
  for (int o = threadIdx.x; o < co; o += 256) {
    float s = 0.f;
    for (int p = 0; p < 256; ++p) s += s_d[o * 256 + p];
    pp[(long long)co * ci * 9 + o] = s;
  }
}

// out[e] = sum_r part[r][e] for e < len (rows in order)
__global__ void k_sum_cols(const float* __restrict__ part, long long ldp, int rows, int len,
                           float* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= len) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += part[(long long)r * ldp + e];
  out[e] = s;
}

// gather the inputs x of the selected samples into act0 [batch][2m][NX]
__global__ void k_gather_x(const float* __restrict__ samples, long long slen, const int* __restrict__ idx,
                           int cx, int NX, float* __restrict__ x) {
  const long long n = (long long)cx * NX;
  const int b = blockIdx.y;
  const float* src = samples + (long long)idx[b] * slen;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    x[(long long)b * n + e] = src[e];
}

// Loss terms and dL/dy at every (sample, pixel).  y [batch][m+m^2][NX]; per sample: t at
// 2m NX, v at 3m NX, w at (3m + S m) NX.  Scales: guess term 1/(m NX), block term
// 1/(S m NX), batch mean 1/batch.
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ samples, long long slen,
                       const int* __restrict__ idx, int m, int S, int NX, int batch, float* __restrict__ dy,
                       double* __restrict__ lpart) {
  __shared__ double red[8];
  const int b = blockIdx.y;
  const int px = blockIdx.x * blockDim.x + threadIdx.x;
  double lsum = 0.0;
  if (px < NX) {
    const int cy = m + m * m;
    const float* yb = y + (long long)b * cy * NX;
    float* db = dy + (long long)b * cy * NX;
    const float* smp = samples + (long long)idx[b] * slen;
    const float* t = smp + 2LL * m * NX;
    const float* v = smp + 3LL * m * NX;
    const float* w = v + (long long)S * m * NX;
    const float sg = 2.f / ((float)m * NX * batch);
    for (int c = 0; c < m; ++c) {
      const float r = yb[(long long)c * NX + px] - t[(long long)c * NX + px];
      lsum += (double)r * r / ((double)m * NX);
      db[(long long)c * NX + px] = sg * r;
    }
    float bm[16];
    for (int e = 0; e < m * m; ++e) bm[e] = yb[(long long)(m + e) * NX + px];
    float gb[16];
    for (int e = 0; e < m * m; ++e) gb[e] = 0.f;
    const float sb = 2.f / ((float)S * m * NX * batch);
    for (int s = 0; s < S; ++s) {
      float ws[4], vs[4];
      for (int c = 0; c < m; ++c) {
        ws[c] = w[((long long)s * m + c) * NX + px];
        vs[c] = v[((long long)s * m + c) * NX + px];
      }
      for (int i = 0; i < m; ++i) {
        float e = ws[i] - vs[i];
        for (int j = 0; j < m; ++j) e = fmaf(bm[i * m + j], ws[j], e);
        lsum += (double)e * e / ((double)S * m * NX);
        for (int j = 0; j < m; ++j) gb[i * m + j] += sb * e * ws[j];
      }
    }
    for (int e = 0; e < m * m; ++e) db[(long long)(m + e) * NX + px] = gb[e];
  }
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    lpart[(long long)b * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void k_loss_fin(const double* lpart, int n, int batch, double* out) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += lpart[i];
  out[0] = s / batch;
}

__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, long long n, float lr, float b1, float b2, float c1,
                       float c2, float eps) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float gv = g[e];
  const float a = b1 * m1[e] + (1.f - b1) * gv;
  const float v = b2 * m2[e] + (1.f - b2) * gv * gv;
  m1[e] = a;
  m2[e] = v;
  th[e] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}

inline unsigned nb(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_conv(const slar_net* net, const float* in, int ci, const float* W, const float* bias,
                        float* out, int co, int batch, int transpose, int ldw_in, int act,
                        const float* gate, cudaStream_t s) {
  dim3 grid(net->tiles, batch);
  switch (net->TW) {
#define CONV_CASE(T)                                                                                  \
  case T:                                                                                             \
    slar::count_launch(), k_conv<T><<<grid, 256, 0, s>>>(in, ci, W, bias, out, co, net->n0, net->n1, \
                                                          transpose, ldw_in, act, gate);              \
    break;
    CONV_CASE(16) CONV_CASE(8) CONV_CASE(4) CONV_CASE(2) CONV_CASE(1)
#undef CONV_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

size_t wgrad_smem(int tw, int ci, int co) { return sizeof(float) * ((size_t)ci * (halo_len(tw) | 1) + (size_t)co * 256); }

cudaError_t launch_wgrad(const slar_net* net, const float* x, int ci, const float* dz, int co, int batch,
                         cudaStream_t s) {
  dim3 grid(net->tiles, batch);
  const size_t sm = wgrad_smem(net->TW, ci, co);
  const long long ldp = (long long)co * ci * 9 + co;
  switch (net->TW) {
#define WG_CASE(T)                                                                             \
  case T:                                                                                      \
    slar::count_launch(), k_conv_wgrad<T><<<grid, 256, sm, s>>>(x, ci, dz, co, net->n0, net->n1, \
                                                                 net->part, ldp);              \
    break;
    WG_CASE(16) WG_CASE(8) WG_CASE(4) WG_CASE(2) WG_CASE(1)
#undef WG_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t init_wgrad_attrs() {
  const int mx = (int)wgrad_smem(1, MAXC, MAXC);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_conv_wgrad<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
  if ((e = cudaFuncSetAttribute(k_conv_wgrad<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
  if ((e = cudaFuncSetAttribute(k_conv_wgrad<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
  if ((e = cudaFuncSetAttribute(k_conv_wgrad<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx))) return e;
  return cudaFuncSetAttribute(k_conv_wgrad<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}

bool pow2(int n) { return n >= 1 && (n & (n - 1)) == 0; }

}  // namespace

// forward pass of `batch` inputs already in net->act[0]; activations kept for backward
cudaError_t net_forward_acts(slar_net* net, int batch, cudaStream_t s) {
  for (int l = 0; l < 4; ++l) {
    cudaError_t e = launch_conv(net, net->act[l], net->cin[l], net->theta + net->woff[l],
                                net->theta + net->boff[l], net->act[l + 1], net->cout[l], batch, 0,
                                net->cin[l], l < 3 ? 1 : 0, nullptr, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// network output for one input x (device FP32 [2m][NX]) on stream s; returns net->act[4]
cudaError_t net_infer(slar_net* net, const float* x, cudaStream_t s, const float** y) {
  cudaError_t e = cudaMemcpyAsync(net->act[0], x, sizeof(float) * 2 * net->m * net->NX,
                                  cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  if ((e = net_forward_acts(net, 1, s)) != cudaSuccess) return e;
  *y = net->act[4];
  return cudaSuccess;
}

int net_m(const slar_net* n) { return n->m; }
int net_nx(const slar_net* n) { return n->NX; }
int net_n0(const slar_net* n) { return n->n0; }
int net_n1(const slar_net* n) { return n->n1; }
long long net_np(const slar_net* n) { return n->np; }

namespace {

long long sample_len(const slar_net* net, int S) { return (3LL * net->m + 2LL * S * net->m) * net->NX; }

// loss (device scalar net->loss_dev) and gradient (net->grad) of the selected samples
cudaError_t loss_grad(slar_net* net, const float* samples, int S, const int* idx, int batch) {
  cudaStream_t s = net->s;
  const int m = net->m, NX = net->NX;
  const long long slen = sample_len(net, S);
  slar::count_launch(), k_gather_x<<<dim3(nb(2LL * m * NX), batch), 256, 0, s>>>(samples, slen, idx, 2 * m, NX,
                                                                                 net->act[0]);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = net_forward_acts(net, batch, s)) != cudaSuccess) return e;
  const int lb = (int)nb(NX);
  slar::count_launch(), k_loss<<<dim3(lb, batch), 256, 0, s>>>(net->act[4], samples, slen, idx, m, S, NX,
                                                               batch, net->dA, net->lpart);
  slar::count_launch(), k_loss_fin<<<1, 32, 0, s>>>(net->lpart, lb * batch, batch, net->loss_dev);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  float* g = net->dA;   // dL/d(pre-activation) of layer l
  float* gnext = net->dB;
  for (int l = 3; l >= 0; --l) {
    if ((e = launch_wgrad(net, net->act[l], net->cin[l], g, net->cout[l], batch, s)) != cudaSuccess) return e;
    const long long len = (long long)net->cout[l] * net->cin[l] * 9 + net->cout[l];
    slar::count_launch(), k_sum_cols<<<nb(len), 256, 0, s>>>(net->part, len, net->tiles * batch, (int)len,
                                                            net->grad + net->woff[l]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (l > 0) {
      // dL/d(pre-activation of layer l-1) = conv^T(g) * (1 - h_{l}^2), h_l = act[l]
      if ((e = launch_conv(net, g, net->cout[l], net->theta + net->woff[l], nullptr, gnext, net->cin[l], batch,
                           1, net->cin[l], 0, net->act[l], s)) != cudaSuccess)
        return e;
      float* t = g;
      g = gnext;
      gnext = t;
    }
  }
  return cudaSuccess;
}

}  // namespace
}  // namespace slar

using namespace slar;

extern "C" slar_status slar_net_param_count(int m, int hidden, long long* out) {
  if (!out || m < 2 || m > 4 || hidden < 1 || hidden > MAXC) return SLAR_EINVAL;
  const int ci[4] = {2 * m, hidden, hidden, hidden};
  const int co[4] = {hidden, hidden, hidden, m + m * m};
  long long n = 0;
  for (int l = 0; l < 4; ++l) n += (long long)co[l] * ci[l] * 9 + co[l];
  *out = n;
  return SLAR_OK;
}

extern "C" slar_status slar_sample_floats(int m, int nx, int n_probes, long long* out) {
  if (!out || m < 2 || m > 4 || nx < 1 || n_probes < 1) return SLAR_EINVAL;
  *out = (3LL * m + 2LL * n_probes * m) * nx;
  return SLAR_OK;
}

extern "C" slar_status slar_net_create(int m, int hidden, int n0, int n1, int max_batch, void* stream,
                                       slar_net** out) {
  if (!out) return SLAR_EINVAL;
  *out = nullptr;
  if (m < 2 || m > 4 || hidden < 1 || hidden > MAXC || !pow2(n0) || !pow2(n1) || n0 > SLAR_MAX_N ||
      n1 > SLAR_MAX_N || max_batch < 1 || max_batch > 4096)
    return SLAR_EINVAL;
  if (m + m * m > MAXC) return SLAR_EINVAL;
  slar_net* net = new slar_net();
  net->m = m;
  net->hidden = hidden;
  net->n0 = n0;
  net->n1 = n1;
  net->NX = n0 * n1;
  net->max_batch = max_batch;
  net->s = static_cast<cudaStream_t>(stream);
  const int ci[4] = {2 * m, hidden, hidden, hidden};
  const int co[4] = {hidden, hidden, hidden, m + m * m};
  long long off = 0;
  for (int l = 0; l < 4; ++l) {
    net->cin[l] = ci[l];
    net->cout[l] = co[l];
    net->woff[l] = off;
    off += (long long)co[l] * ci[l] * 9;
    net->boff[l] = off;
    off += co[l];
  }
  net->np = off;
  net->TW = n1 < 16 ? n1 : 16;
  net->TH = 256 / net->TW;
  net->tiles = ((n0 + net->TH - 1) / net->TH) * ((n1 + net->TW - 1) / net->TW);
  const long long NX = net->NX;
  long long maxc = 2 * m;
  for (int l = 0; l < 4; ++l) maxc = std::max<long long>(maxc, co[l]);
  net->part_len = (long long)net->tiles * max_batch * (MAXC * MAXC * 9 + MAXC);
  bool ok = cudaMalloc(&net->theta, sizeof(float) * net->np) == cudaSuccess &&
            cudaMalloc(&net->grad, sizeof(float) * net->np) == cudaSuccess &&
            cudaMalloc(&net->am, sizeof(float) * net->np) == cudaSuccess &&
            cudaMalloc(&net->av, sizeof(float) * net->np) == cudaSuccess &&
            cudaMalloc(&net->dA, sizeof(float) * maxc * NX * max_batch) == cudaSuccess &&
            cudaMalloc(&net->dB, sizeof(float) * maxc * NX * max_batch) == cudaSuccess &&
            cudaMalloc(&net->part, sizeof(float) * net->part_len) == cudaSuccess &&
            cudaMalloc(&net->lpart, sizeof(double) * (nb(NX) * (long long)max_batch + 1)) == cudaSuccess &&
            cudaMalloc(&net->loss_dev, sizeof(double)) == cudaSuccess &&
            cudaMallocHost(&net->loss_host, sizeof(double)) == cudaSuccess;
  const int chans[5] = {2 * m, hidden, hidden, hidden, m + m * m};
  for (int l = 0; l < 5 && ok; ++l)
    ok = cudaMalloc(&net->act[l], sizeof(float) * chans[l] * NX * max_batch) == cudaSuccess;
  if (ok) ok = init_wgrad_attrs() == cudaSuccess;
  if (ok) ok = cudaMemsetAsync(net->theta, 0, sizeof(float) * net->np, net->s) == cudaSuccess &&
               cudaMemsetAsync(net->am, 0, sizeof(float) * net->np, net->s) == cudaSuccess &&
               cudaMemsetAsync(net->av, 0, sizeof(float) * net->np, net->s) == cudaSuccess;
  if (!ok) {
    slar_net_destroy(net);
    return SLAR_ENOMEM;
  }
  *out = net;
  return SLAR_OK;
}

extern "C" slar_status slar_net_destroy(slar_net* net) {
  if (!net) return SLAR_OK;
  if (net->s || true) cudaStreamSynchronize(net->s);
  float* fs[] = {net->theta, net->grad, net->am, net->av, net->dA, net->dB, net->part,
                 net->act[0], net->act[1], net->act[2], net->act[3], net->act[4]};
  for (float* p : fs)
    if (p) cudaFree(p);
  if (net->lpart) cudaFree(net->lpart);
  if (net->loss_dev) cudaFree(net->loss_dev);
  if (net->loss_host) cudaFreeHost(net->loss_host);
  delete net;
  return SLAR_OK;
}

extern "C" slar_status slar_net_set_params(slar_net* net, const float* theta, long long n) {
  if (!net || !theta || n != net->np) return SLAR_EINVAL;
  if (cudaMemcpyAsync(net->theta, theta, sizeof(float) * n, cudaMemcpyHostToDevice, net->s) != cudaSuccess ||
      cudaMemsetAsync(net->am, 0, sizeof(float) * n, net->s) != cudaSuccess ||
      cudaMemsetAsync(net->av, 0, sizeof(float) * n, net->s) != cudaSuccess ||
      cudaStreamSynchronize(net->s) != cudaSuccess)
    return SLAR_ECUDA;
  net->t = 0;
  return SLAR_OK;
}

extern "C" slar_status slar_net_get_params(slar_net* net, float* theta, long long n) {
  if (!net || !theta || n != net->np) return SLAR_EINVAL;
  if (cudaMemcpyAsync(theta, net->theta, sizeof(float) * n, cudaMemcpyDeviceToHost, net->s) != cudaSuccess ||
      cudaStreamSynchronize(net->s) != cudaSuccess)
    return SLAR_ECUDA;
  return SLAR_OK;
}

extern "C" slar_status slar_net_forward(slar_net* net, const float* x, int batch, float* y) {
  if (!net || !x || !y || batch < 1 || batch > net->max_batch) return SLAR_EINVAL;
  const long long nin = 2LL * net->m * net->NX * batch;
  const long long nout = (long long)(net->m + net->m * net->m) * net->NX * batch;
  if (cudaMemcpyAsync(net->act[0], x, sizeof(float) * nin, cudaMemcpyDeviceToDevice, net->s) != cudaSuccess)
    return SLAR_ECUDA;
  if (net_forward_acts(net, batch, net->s) != cudaSuccess) return SLAR_ECUDA;
  if (cudaMemcpyAsync(y, net->act[4], sizeof(float) * nout, cudaMemcpyDeviceToDevice, net->s) != cudaSuccess)
    return SLAR_ECUDA;
  return SLAR_OK;
}

extern "C" slar_status slar_net_loss_grad(slar_net* net, const float* samples, int S, const int* idx, int batch,
                                          double* loss, float* grad) {
  if (!net || !samples || !idx || S < 1 || batch < 1 || batch > net->max_batch) return SLAR_EINVAL;
  if (loss_grad(net, samples, S, idx, batch) != cudaSuccess) return SLAR_ECUDA;
  if (grad && cudaMemcpyAsync(grad, net->grad, sizeof(float) * net->np, cudaMemcpyDeviceToDevice, net->s) !=
                  cudaSuccess)
    return SLAR_ECUDA;
  if (loss) {
    if (cudaMemcpyAsync(net->loss_host, net->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, net->s) !=
            cudaSuccess ||
        cudaStreamSynchronize(net->s) != cudaSuccess)
      return SLAR_ECUDA;
    *loss = net->loss_host[0];
  }
  return SLAR_OK;
}

extern "C" slar_status slar_net_train_step(slar_net* net, const float* samples, int S, const int* idx, int batch,
                                           float lr, double* loss) {
  if (!net || !samples || !idx || S < 1 || batch < 1 || batch > net->max_batch || !(lr > 0.f))
    return SLAR_EINVAL;
  if (loss_grad(net, samples, S, idx, batch) != cudaSuccess) return SLAR_ECUDA;
  net->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = (float)(1.0 - std::pow(0.9, (double)net->t));
  const float c2 = (float)(1.0 - std::pow(0.999, (double)net->t));
  slar::count_launch(), k_adam<<<nb(net->np), 256, 0, net->s>>>(net->theta, net->grad, net->am, net->av, net->np,
                                                               lr, b1, b2, c1, c2, 1e-8f);
  if (cudaGetLastError() != cudaSuccess) return SLAR_ECUDA;
  if (loss) {
    if (cudaMemcpyAsync(net->loss_host, net->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, net->s) !=
            cudaSuccess ||
        cudaStreamSynchronize(net->s) != cudaSuccess)
      return SLAR_ECUDA;
    *loss = net->loss_host[0];
  }
  return SLAR_OK;
}
