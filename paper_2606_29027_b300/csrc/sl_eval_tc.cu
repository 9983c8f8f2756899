// Entry evaluator whose transfer-tensor contractions (Sec. 3.1, the O(d r^3) part of an
// entry, Eq. tp_interp in HT form) run on the 5th-generation tensor cores: tcgen05.mma,
// kind::f16 with BF16 operands and FP32 accumulation in tensor memory, in the BF16x3 split
// x = hi + lo (hi = bf16(x), lo = bf16(x - hi)), a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi.
// Trees with d = 4 only (a d = 2 tree has no transfer tensor).
//
// One CTA evaluates 128 entries (the MMA's M):
//   1. feet and quadratic weights (FP32, shared with the FP32 SIMT evaluator),
//   2. leaf gathers c^(mu) (FP32) for the two children of the node,
//   3. c_t[e][p] = sum_k KR[e][k] B_t[p][k], k = (a, b), KR[e][(a,b)] = c1[e][a] c2[e][b]:
//      a [128 x K] x [K x N] GEMM.  Per K-chunk of 64 the CTA writes KR (hi, lo) into
//      shared memory and copies the pre-split chunk of B_t (hi, lo); one thread issues
//      3 x 4 MMAs (K-steps of 16) into the node's TMEM accumulator and commits them to an
//      mbarrier, which every thread waits on (bounded) before the buffers are reused,
//   4. the root contraction, correction and residual epilogue as in the SIMT evaluator.
// Shared-memory operand layout (canonical, no swizzle, K-major): K-step s | 8-row group |
// K core matrix | 8 rows x 16 bytes; byte (row, kk) = (row / 8) 256 + (kk / 8) 128 +
// (row % 8) 16 + (kk % 8) 2 for kk < 16, i.e. leading (K) byte offset 128, stride (M/N)
// byte offset 256.  Every address the descriptors can form lies inside its 16-row-group
// tile whichever of the two offsets the hardware applies along K.
#include <cuda_bf16.h>

#include "common.cuh"
#include "eval_device.cuh"

namespace slar {
namespace {

constexpr int TC_TILE = 128;
constexpr int TC_THREADS = 256;
constexpr int TC_TMEM_COLS = 128;          // two accumulators of <= 64 columns
constexpr long long TC_WAIT_LIMIT = 1LL << 22;
constexpr int TC_HEAD_BYTES = 23552;       // feet, weights, values (FP64) and rows (int)
constexpr int TC_A_BYTES = 32768;          // KR chunk: 2 parts x 4 K-steps x 4096 B

__host__ __device__ __forceinline__ int tc_np(int rp) {
  const int n = ((rp + 15) / 16) * 16;
  return n < 16 ? 16 : n;
}
__host__ __device__ __forceinline__ int tc_chunk_bytes(int np) { return 256 * np; }
__host__ __device__ __forceinline__ int al128(int x) { return (x + 127) & ~127; }

struct TcLayout {
  int ca, cb, c12, c34, A, B, total;
};

__host__ __device__ __forceinline__ TcLayout tc_layout(int r0, int r1, int r2, int r3, int r12, int r34) {
  TcLayout L;
  const int ra = r0 > r2 ? r0 : r2, rb = r1 > r3 ? r1 : r3;
  const int np = tc_np(r12) > tc_np(r34) ? tc_np(r12) : tc_np(r34);
  int o = TC_HEAD_BYTES;
  L.ca = o; o = al128(o + 4 * TC_TILE * (ra + 1));
  L.cb = o; o = al128(o + 4 * TC_TILE * (rb + 1));
  L.c12 = o; o = al128(o + 4 * TC_TILE * r12);
  L.c34 = o; o = al128(o + 4 * TC_TILE * r34);
  L.A = o; o += TC_A_BYTES;
  L.B = o; o += 2 * tc_chunk_bytes(np);   // double buffer
  L.total = o;
  return L;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start address, leading byte offset 128, stride byte
// offset 256, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
         ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void split8(const float* x, uint4* hi, uint4* lo) {
  __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    h[j] = __float2bfloat16_rn(x[j]);
    l[j] = __float2bfloat16_rn(x[j] - __bfloat162float(h[j]));
  }
  *hi = *reinterpret_cast<uint4*>(h);
  *lo = *reinterpret_cast<uint4*>(l);
}

// asynchronous copy of one pre-split chunk (bytes a multiple of 16) into shared memory,
// one commit group per chunk
__device__ __forceinline__ void copy_chunk_async(unsigned char* dst, const unsigned char* src, int bytes) {
  const uint32_t d = smem_u32(dst);
  for (int it = threadIdx.x; it < bytes / 16; it += TC_THREADS)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + 16 * it), "l"(src + 16LL * it) : "memory");
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// Pre-split B [rp][K] (FP32, row = p) into per-chunk hi/lo operand tiles (layout above).
__global__ void k_split_bf16(const float* __restrict__ B, int rp, int K, int np, int nch,
                             unsigned char* __restrict__ out) {
  const long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= (long long)nch * np * 8) return;
  const int c = (int)(it / (np * 8));
  const int r = (int)(it % (np * 8));
  const int p = r >> 3, kg = r & 7;
  float x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int k = c * 64 + kg * 8 + j;
    x[j] = (p < rp && k < K) ? B[(long long)p * K + k] : 0.f;
  }
  uint4 hi, lo;
  split8(x, &hi, &lo);
  unsigned char* base = out + (long long)c * tc_chunk_bytes(np);
  const int off = (kg >> 1) * 32 * np + (p >> 3) * 256 + (kg & 1) * 128 + (p & 7) * 16;
  *reinterpret_cast<uint4*>(base + off) = hi;
  *reinterpret_cast<uint4*>(base + 128 * np + off) = lo;
}

// c_out[e][p] = sum_{a,b} ca[e][a] cb[e][b] B[p][a][b] on the tensor cores; returns false
// (with *err set) if an MMA completion wait ran out.
__device__ bool contract_tc(const float* ca, int ra, const float* cb, int rb, const unsigned char* Bg, int rp,
                            float* cout, uint32_t tmem_d, unsigned char* Abuf, unsigned char* Bbuf, uint32_t bar,
                            uint32_t& phase, int nT, int* s_ok, int* err) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = ra * rb, np = tc_np(rp), nch = (K + 63) / 64;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(np >> 3) << 17) |
                         ((uint32_t)(TC_TILE >> 4) << 24);
  const uint32_t a_addr = smem_u32(Abuf);
  const int cb_bytes = tc_chunk_bytes(np);
  copy_chunk_async(Bbuf, Bg, cb_bytes);   // chunk 0 into buffer 0
  for (int c = 0; c < nch; ++c) {
    // prefetch chunk c+1 into the other buffer (its previous MMA has completed)
    if (c + 1 < nch) copy_chunk_async(Bbuf + ((c + 1) & 1) * cb_bytes, Bg + (long long)(c + 1) * cb_bytes, cb_bytes);
    // Khatri-Rao chunk of the left operand, split into hi / lo.  A warp takes 32
    // consecutive entries of one 8-wide k-group: its 16-byte stores fill whole 128-byte
    // rows of core matrices (no bank conflicts), its reads of ca / cb use the odd padded
    // strides, and (a, b) of the group's first k is the same across the warp.
    const int lda = ra + 1, ldb = rb + 1;
    for (int it = tid; it < TC_TILE * 8; it += TC_THREADS) {
      const int kg = it >> 7, e = it & (TC_TILE - 1);
      const int k0 = c * 64 + kg * 8;
      int a = k0 / rb, b = k0 - a * rb;
      const bool live = e < nT;
      const float* cae = ca + e * lda;
      const float* cbe = cb + e * ldb;
      float x[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        x[j] = (live && k0 + j < K) ? cae[a] * cbe[b] : 0.f;
        if (++b == rb) {
          b = 0;
          ++a;
        }
      }
      uint4 hi, lo;
      split8(x, &hi, &lo);
      const int off = (kg >> 1) * 4096 + (e >> 3) * 256 + (kg & 1) * 128 + (e & 7) * 16;
      *reinterpret_cast<uint4*>(Abuf + off) = hi;
      *reinterpret_cast<uint4*>(Abuf + 16384 + off) = lo;
    }
    // chunk c's copy done (chunk c+1 may still be in flight)
    if (c + 1 < nch) asm volatile("cp.async.wait_group 1;" ::: "memory");
    else asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      fence_after();
      const uint32_t b_addr = smem_u32(Bbuf + (c & 1) * cb_bytes);
      for (int s = 0; s < 4; ++s) {
        if (c * 64 + s * 16 >= K) break;
        const uint64_t ah = tc_desc(a_addr + s * 4096), al = tc_desc(a_addr + 16384 + s * 4096);
        const uint64_t bh = tc_desc(b_addr + s * 32 * np), bl = tc_desc(b_addr + 128 * np + s * 32 * np);
        mma_bf16(tmem_d, ah, bh, idesc, (c > 0 || s > 0) ? 1u : 0u);
        mma_bf16(tmem_d, ah, bl, idesc, 1u);
        mma_bf16(tmem_d, al, bh, idesc, 1u);
      }
      mma_commit(bar);
      long long n = 0;
      bool ok = mbar_try_wait(bar, phase);
      while (!ok && ++n < TC_WAIT_LIMIT) ok = mbar_try_wait(bar, phase);
      if (!ok) {
        atomicExch(err, 1);
        n = 0;
        while (!mbar_try_wait(bar, phase) && ++n < TC_WAIT_LIMIT) {
        }
        *s_ok = 0;
      }
    }
    phase ^= 1u;
    __syncthreads();
    if (!*s_ok) {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      return false;
    }
  }
  fence_after();
  if (warp < 4) {
    const int e = 32 * warp + lane;
    for (int j0 = 0; j0 < np; j0 += 16) {
      uint32_t r[16];
      tmem_ld16(tmem_d + ((uint32_t)(32 * warp) << 16) + (uint32_t)j0, r);
      if (e < nT)
#pragma unroll
        for (int jj = 0; jj < 16; ++jj)
          if (j0 + jj < rp) cout[e * rp + j0 + jj] = __uint_as_float(r[jj]);
    }
  }
  fence_before();
  __syncthreads();
  return true;
}

template <bool DEV>
__global__ void __launch_bounds__(TC_THREADS)
k_sl_eval_tc(GridDesc g, HTView<float> ht_arg, CorrView corr_arg, const EvalParams<float>* __restrict__ P,
             EvalArgs a, const unsigned char* __restrict__ b12, const unsigned char* __restrict__ b34, int* err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long s_bar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_ok;
  HTView<float> ht;
  CorrView corr;
  if (DEV) {
    const EvalParams<float> q = *P;
    ht = q.ht;
    corr = q.corr;
    a.tau = q.tau;
    a.E = q.E;
    a.foot_euler = q.foot_euler;
  } else {
    ht = ht_arg;
    corr = corr_arg;
  }
  if (a.done && *a.done) return;
  if (a.kidx) {
    const int kk = *a.kidx;
    a.pivot += kk;
    a.kterms = kk;
    a.out += kk * a.out_stride;
  }
  const long long e0 = (long long)blockIdx.x * TC_TILE;
  if (e0 >= a.n) return;
  const int nT = (int)min((long long)TC_TILE, a.n - e0);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int d = g.d;
  const TcLayout L = tc_layout(ht.r[0], ht.r[1], ht.r[2], ht.r[3], ht.r12, ht.r34);
  double* sfoot = reinterpret_cast<double*>(smem_raw);   // 128 x 4
  double* sw = sfoot + TC_TILE * 4;                       // 128 x 12
  double* sval = sw + TC_TILE * 12;                       // 128
  int* srow = reinterpret_cast<int*>(sval + TC_TILE);     // 128 x 12
  float* ca = reinterpret_cast<float*>(smem_raw + L.ca);
  float* cb = reinterpret_cast<float*>(smem_raw + L.cb);
  float* c12 = reinterpret_cast<float*>(smem_raw + L.c12);
  float* c34 = reinterpret_cast<float*>(smem_raw + L.c34);
  unsigned char* Abuf = smem_raw + L.A;
  unsigned char* Bbuf = smem_raw + L.B;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_ok = 1;
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t bar = smem_u32(&s_bar);
  uint32_t phase = 0;

  // 1. feet and weights
  if (tid < nT) {
    int idx[4];
    decode_tuple(g, a, e0 + tid, idx);
    float foot[4];
    trace_foot_f(g, a.E, a.tau, a.foot_euler, idx, foot);
    for (int m = 0; m < d; ++m) {
      int r[3];
      float w[3];
      cell_weights_f(g, m, foot[m], r, w);
      for (int s = 0; s < 3; ++s) {
        srow[(tid * 4 + m) * 3 + s] = r[s];
        sw[(tid * 4 + m) * 3 + s] = w[s];
      }
      sfoot[tid * 4 + m] = foot[m];
    }
  }
  __syncthreads();

  bool ok = true;
  for (int node = 0; node < 2 && ok; ++node) {
    // 2. leaf gathers of the node's two children
    for (int side = 0; side < 2; ++side) {
      const int m = 2 * node + side;
      const int r = ht.r[m];
      const float* U = ht.U[m];
      float* c = side == 0 ? ca : cb;
      for (int it = tid; it < TC_TILE * r; it += TC_THREADS) {
        const int t = it / r, q = it - t * r;
        float val = 0.f;
        if (t < nT) {
          const int* rr = srow + (t * 4 + m) * 3;
          const double* ww = sw + (t * 4 + m) * 3;
          val = (float)ww[0] * U[(long long)rr[0] * r + q] + (float)ww[1] * U[(long long)rr[1] * r + q] +
                (float)ww[2] * U[(long long)rr[2] * r + q];
        }
        c[t * (r + 1) + q] = val;   // odd row stride (conflict-free reads across entries)
      }
    }
    __syncthreads();
    // 3. transfer tensor on the tensor cores
    ok = node == 0 ? contract_tc(ca, ht.r[0], cb, ht.r[1], b12, ht.r12, c12, tmem, Abuf, Bbuf, bar, phase, nT,
                                 &s_ok, err)
                   : contract_tc(ca, ht.r[2], cb, ht.r[3], b34, ht.r34, c34, tmem + 64, Abuf, Bbuf, bar, phase,
                                 nT, &s_ok, err);
  }

  if (ok) {
    // 4. root: sum_p c12[t][p] sum_q Broot[p][q] c34[t][q]
    constexpr int TPE = TC_THREADS / TC_TILE;
    const int t = tid / TPE, sub = tid - t * TPE;
    const int rl = ht.r12, rr = ht.r34;
    float acc = 0.f;
    if (t < nT) {
      for (int p = sub; p < rl; p += TPE) {
        float s = 0.f;
        const float* Bp = ht.Broot + (long long)p * rr;
        for (int q = 0; q < rr; ++q) s += Bp[q] * c34[t * rr + q];
        acc += c12[t * rl + p] * s;
      }
    }
#pragma unroll
    for (int off = TPE / 2; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off, TPE);
    if (sub == 0 && t < TC_TILE) sval[t] = (double)acc;
    __syncthreads();
    // 5. correction and residual epilogue
    if (tid < nT) {
      double val = sval[tid];
      if (corr.has) {
        float f4[4];
        for (int m = 0; m < d; ++m) f4[m] = (float)sfoot[tid * 4 + m];
        val += (double)correction_at_f(g, corr, f4);
      }
      const long long e = e0 + tid;
      if (a.X) {
        const long long piv = (long long)(*a.pivot);
        for (int l = 0; l < a.kterms; ++l) val -= a.X[piv + l * a.ldX] * a.Y[e + l * a.ldY];
      }
      a.out[e] = val;
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                 : "memory");
  }
}

}  // namespace

size_t sl_eval_tc_smem(const int* r6) {
  return (size_t)tc_layout(r6[0], r6[1], r6[2], r6[3], r6[4], r6[5]).total;
}

long long tc_split_bytes() { return 64LL * tc_chunk_bytes(64); }

cudaError_t sl_eval_tc_init_attrs() {
  const int mx = 220 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_sl_eval_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sl_eval_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  return e;
}

cudaError_t split_transfer_bf16(const float* B, int rp, int ra, int rb, void* out, cudaStream_t s) {
  const int K = ra * rb, np = tc_np(rp), nch = (K + 63) / 64;
  if (rp > 64 || nch > 64) return cudaErrorInvalidValue;
  const long long n = (long long)nch * np * 8;
  slar::count_launch(), k_split_bf16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(B, rp, K, np, nch,
                                                                                static_cast<unsigned char*>(out));
  return cudaGetLastError();
}

cudaError_t launch_sl_eval_tc(const GridDesc& g, const HTView<float>& ht, const CorrView& corr, const EvalArgs& a,
                              const void* b12, const void* b34, int* err, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  if (g.d != 4) return cudaErrorInvalidValue;
  const int r6[6] = {ht.r[0], ht.r[1], ht.r[2], ht.r[3], ht.r12, ht.r34};
  const size_t sm = sl_eval_tc_smem(r6);
  const long long blocks = (a.n + TC_TILE - 1) / TC_TILE;
  slar::count_launch(), k_sl_eval_tc<false><<<(unsigned)blocks, TC_THREADS, sm, s>>>(
      g, ht, corr, nullptr, a, static_cast<const unsigned char*>(b12), static_cast<const unsigned char*>(b34), err);
  return cudaGetLastError();
}

cudaError_t launch_sl_eval_tc_dev(const GridDesc& g, const EvalParams<float>* P, const EvalArgs& a, const void* b12,
                                  const void* b34, int* err, size_t sm, cudaStream_t s) {
  if (g.d != 4) return cudaErrorInvalidValue;
  const long long blocks = (a.n + TC_TILE - 1) / TC_TILE;
  slar::count_launch(), k_sl_eval_tc<true><<<(unsigned)blocks, TC_THREADS, sm, s>>>(
      g, HTView<float>{}, CorrView{}, P, a, static_cast<const unsigned char*>(b12),
      static_cast<const unsigned char*>(b34), err);
  return cudaGetLastError();
}

}  // namespace slar
