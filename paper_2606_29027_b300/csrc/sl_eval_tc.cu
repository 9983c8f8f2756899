// Entry evaluator whose transfer-tensor contractions (Sec. 3.1, the O(d r^3) part of an
// entry, Eq. tp_interp in HT form) run on the 5th-generation tensor cores: tcgen05.mma,
// kind::f16 with BF16 operands and FP32 accumulation in tensor memory, in one of two splits:
//   BF16x3  x = hi + lo (hi = bf16(x), lo = bf16(x - hi)), a b ~ a_hi b_hi + a_hi b_lo +
//           a_lo b_hi (three products, the dropped a_lo b_lo ~ 2^-16 |a b|),
//   BF16x6  x = x1 + x2 + x3 (each the BF16 rounding of what is left), a b ~ the six
//           products a_i b_j with i + j <= 4 (the dropped ones ~ 2^-24 |a b|, FP32's own
//           rounding), 128-column chunks becoming 64-column ones (see below).
// Trees with d = 4 only (a d = 2 tree has no transfer tensor).
//
// A transfer node t with children (mu1, mu2) maps the leaf rows c1 = c^(mu1)[e][.],
// c2 = c^(mu2)[e][.] to c_t[e][p] = sum_a c1[e][a] sum_b B_t[p][a][b] c2[e][b].  One CTA
// evaluates 128 entries (the MMA's M) in two stages per node:
//   T[e][(p, a)] = sum_b c2[e][b] B_t[p][a][b]        a [128 x rb] x [rb x rp ra] GEMM on
//                                                      the tensor cores (K = rb),
//   c_t[e][p]    = sum_a c1[e][a] T[e][(p, a)]        per-entry dot products on the CUDA
//                                                      cores, reading T from tensor memory.
// The columns (p, a) of both nodes (a padded to ra16, a multiple of 16) form one stream of
// chunks of W columns (W = 128 for BF16x3, each chunk an even number of whole p; W = 64 for
// BF16x6, whole p, and at ra16 > 32 one p per chunk).  Three warp roles run the stream
// through a 3-stage ring:
//   warp 9 (one thread)   bulk-copies chunk j's pre-split B tile (all pieces) into shared
//                         slot j % 3 once the MMAs of chunk j - 3 have released it,
//   warp 8 (one thread)   issues chunk j's 3 (6) x K/16 MMAs into tensor-memory slot j % 3
//                         once the tile has landed and chunk j - 3 has been read out, and
//                         commits them to an mbarrier,
//   warps 0-7             read chunk j out of tensor memory (one load of W/2 columns per
//                         warp: the warp pair of a lane quadrant splits the chunk's columns
//                         in halves), dot them with c1 held in registers and store c_t[e][p]
//                         as a tensor-memory column; each warp then arrives on the slot's
//                         mbarrier.  A BF16x6 p split across the two halves leaves two
//                         partial sums, added before the root contraction.
// c2 of both nodes is the MMA's A operand (gathered and split once per CTA), c1 of the
// current node sits in registers (the thread's own entry), and c_12, c_34 stay in tensor
// memory for the root contraction and the correction / residual epilogue of the SIMT
// evaluator.
// Shared-memory operand layout (canonical, no swizzle, K-major): K-step s | 8-row group |
// K core matrix | 8 rows x 16 bytes; byte (row, kk) = (row / 8) 256 + (kk / 8) 128 +
// (row % 8) 16 + (kk % 8) 2 for kk < 16, i.e. leading (K) byte offset 128, stride (M/N)
// byte offset 256.
// Every wait is bounded: a wait that runs out sets *err, the CTA skips the remaining work,
// waits (bounded) for its copies and MMAs in flight and frees its tensor memory.
#include <cuda_bf16.h>

#include "common.cuh"
#include "eval_device.cuh"

namespace slar {
namespace {

constexpr int TC_TILE = 128;
constexpr int TC_CONSUMERS = 256;        // warps 0-7
constexpr int TC_MMA_WARP = 8;
constexpr int TC_COPY_WARP = 9;
constexpr int TC_THREADS = 320;
constexpr int TC_STAGES = 3;
constexpr int TC_TMEM_COLS = 512;        // 3 chunk slots, c_12 and c_34 (and their second halves)

// Operands split into PC BF16 pieces: PC = 2 (x = hi + lo, three products hh + hl + lh, about
// 2^-16 relative per product) or PC = 3 (x = x1 + x2 + x3, six products 11 + 12 + 21 + 13 + 31
// + 22, about 2^-24).  Columns per chunk: 128 with two pieces; 64 with three, so that the
// ring of three 1.5x larger B slots and the 1.5x larger A tiles fit in shared memory at rank
// 64.  Tensor-memory columns: three chunk slots, then c_12 and c_34; with three pieces the
// read-out of a p whose a-range spans both 32-column halves of a chunk leaves two partial
// sums, the second in the columns after c_34 (c_12b, c_34b).
template <int PC> __host__ __device__ constexpr int tc_w() { return PC == 2 ? 128 : 64; }
template <int PC> __host__ __device__ constexpr int tc_out12() { return 3 * tc_w<PC>(); }
template <int PC> __host__ __device__ constexpr int tc_out34() { return 3 * tc_w<PC>() + 64; }
template <int PC> __host__ __device__ constexpr int tc_out12b() { return 3 * tc_w<PC>() + 128; }
template <int PC> __host__ __device__ constexpr int tc_out34b() { return 3 * tc_w<PC>() + 192; }
constexpr long long TC_WAIT_LIMIT = 1LL << 22;
constexpr int TC_HEAD_BYTES = 2048;      // values and partial sums of the root
constexpr int PRO_HEAD_BYTES = 16384;    // prologue: feet, weights, rows
constexpr int TC_MIN_SMEM = 120 * 1024;  // one CTA per SM: the 512-column allocation never waits

__host__ __device__ __forceinline__ int r16(int r) { return ((r + 15) / 16) * 16; }
template <int PC>
__host__ __device__ __forceinline__ int tc_width(int ra16) { return (tc_w<PC>() / ra16) * ra16; }
__host__ __device__ __forceinline__ int al128(int x) { return (x + 127) & ~127; }
__host__ __device__ __forceinline__ int stage_ld(int r) { return r | 1; }   // odd row stride

struct TcLayout {
  int A0, A1, B, slot, rootB, total;
};

template <int PC>
__host__ __device__ __forceinline__ TcLayout tc_layout(int r0, int r1, int r2, int r3, int r12, int r34) {
  TcLayout L;
  (void)r0;
  (void)r2;
  int o = TC_HEAD_BYTES;
  L.A0 = o; o += TC_TILE * r16(r1) * 2 * PC;
  L.A1 = o; o += TC_TILE * r16(r3) * 2 * PC;
  const int s0 = tc_width<PC>(r16(r0)) * r16(r1) * 2 * PC, s1 = tc_width<PC>(r16(r2)) * r16(r3) * 2 * PC;
  L.slot = s0 > s1 ? s0 : s1;
  L.B = o; o += TC_STAGES * L.slot;
  // the root contraction reuses the A and B regions once the chunk stream is over: its A
  // operand (c34, 128 x r34) at A0, the pre-split Broot after it
  L.rootB = al128(L.A0 + TC_TILE * r16(r34) * 2 * PC);
  const int root_end = L.rootB + r16(r12) * r16(r34) * 2 * PC;
  if (root_end > o) o = root_end;
  L.total = o > TC_MIN_SMEM ? o : TC_MIN_SMEM;
  return L;
}

// one transfer node as the chunk stream sees it
struct TcNode {
  int ra, rp, ra16, rb16, ks, w, pc, ntot, nch, out_col;
  uint32_t a_addr;                 // A operand (c2 split) in shared memory
  const unsigned char* bg;         // pre-split B tiles in global memory
};

template <int PC>
__device__ __forceinline__ TcNode tc_node(int ra, int rb, int rp, uint32_t a_addr, const unsigned char* bg,
                                          int out_col) {
  TcNode n;
  n.ra = ra; n.rp = rp;
  n.ra16 = r16(ra); n.rb16 = r16(rb); n.ks = n.rb16 / 16;
  n.w = tc_width<PC>(n.ra16); n.pc = n.w / n.ra16;
  n.ntot = rp * n.ra16; n.nch = (n.ntot + n.w - 1) / n.w;
  n.out_col = out_col;
  n.a_addr = a_addr;
  n.bg = bg;
  return n;
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

__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
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

// bounded wait of one thread
__device__ __forceinline__ bool wait_one_n(uint32_t bar, uint32_t parity, long long limit) {
  for (long long n = 0; n < limit; ++n)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ bool wait_one(uint32_t bar, uint32_t parity) {
  return wait_one_n(bar, parity, TC_WAIT_LIMIT);
}

// bounded wait of a whole warp: true on every lane once every lane has seen the phase
__device__ __forceinline__ bool wait_warp(uint32_t bar, uint32_t parity) {
  bool ok = false;
  for (long long n = 0; n < TC_WAIT_LIMIT; ++n) {
    ok = ok || mbar_try_wait(bar, parity);
    if (__all_sync(0xffffffffu, ok)) return true;
  }
  return false;
}

// bulk copy global -> shared, completion counted in bytes on the mbarrier
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float* v) {
  uint32_t* r = reinterpret_cast<uint32_t*>(v);
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t* r = reinterpret_cast<uint32_t*>(v);
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t* r = reinterpret_cast<uint32_t*>(v);
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_st1(uint32_t taddr, float v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(taddr), "r"(__float_as_uint(v)) : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// x = piece 0 + piece 1 (+ piece 2), each the BF16 rounding of what the earlier pieces leave
template <int PC>
__device__ __forceinline__ void split8(const float* x, uint4* out) {
  __align__(16) __nv_bfloat16 h[PC][8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float rest = x[j];
#pragma unroll
    for (int q = 0; q < PC; ++q) {
      h[q][j] = __float2bfloat16_rn(rest);
      rest -= __bfloat162float(h[q][j]);
    }
  }
#pragma unroll
  for (int q = 0; q < PC; ++q) out[q] = *reinterpret_cast<uint4*>(h[q]);
}

// Pre-split B [rp][ra][b] (FP32) into the chunk tiles of the column stream: row n = (p, a)
// (a padded to ra16), K = b (padded to rb16); chunk c holds rows [c W, c W + Wc) as
// [hi: ks K-step tiles of Wc x 16][lo: same], tile layout as above.
template <int PC>
__global__ void k_split_bf16(const float* __restrict__ B, int rp, int ra, int rb, unsigned char* __restrict__ out) {
  const int ra16 = r16(ra), rb16 = r16(rb), ks = rb16 / 16, W = tc_width<PC>(ra16), ntot = rp * ra16, ng = rb16 / 8;
  const long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= (long long)ntot * ng) return;
  const int n = (int)(it / ng), kg = (int)(it % ng);
  const int p = n / ra16, a = n - p * ra16;
  float x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int b = kg * 8 + j;
    x[j] = (a < ra && b < rb) ? B[((long long)p * ra + a) * rb + b] : 0.f;
  }
  uint4 pc[PC];
  split8<PC>(x, pc);
  const int cl = n / W, nl = n - cl * W;
  const int wc = min(W, ntot - cl * W);
  unsigned char* base = out + (long long)cl * W * rb16 * 2 * PC;
  const int off = (kg >> 1) * wc * 32 + (nl >> 3) * 256 + (kg & 1) * 128 + (nl & 7) * 16;
#pragma unroll
  for (int q = 0; q < PC; ++q) *reinterpret_cast<uint4*>(base + q * ks * wc * 32 + off) = pc[q];
}

// stage[e][q] = sum_s w[e][m][s] U_m[row_s][q] (FP32), zero rows for e >= nT.  Lanes run
// over q (coalesced reads of U, conflict-free writes with the odd stride); each thread
// issues the loads of four items before it uses them.
__device__ __forceinline__ void gather_leaf(float* stage, const float* __restrict__ U, int r, int m, int nT,
                                            const int* srow, const float* sw) {
  const int ld = stage_ld(r), n = TC_TILE * r;
  for (int base = threadIdx.x; base < n; base += 4 * TC_THREADS) {
    float u[4][3], w[4][3];
    int dst[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int it = base + k * TC_THREADS;
      dst[k] = -1;
      u[k][0] = u[k][1] = u[k][2] = 0.f;
      w[k][0] = w[k][1] = w[k][2] = 0.f;
      if (it < n) {
        const int e = it / r, q = it - e * r;
        dst[k] = e * ld + q;
        if (e < nT) {
          const int* rr = srow + (e * 4 + m) * 3;
          const float* ww = sw + (e * 4 + m) * 3;
#pragma unroll
          for (int s = 0; s < 3; ++s) {
            u[k][s] = __ldg(U + (long long)rr[s] * r + q);
            w[k][s] = ww[s];
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (dst[k] >= 0) stage[dst[k]] = w[k][0] * u[k][0] + w[k][1] * u[k][1] + w[k][2] * u[k][2];
  }
}

// Pre-split Broot [r12][r34] (FP32) into the B operand of the root contraction: rows n = p
// (N = r12 padded to 16), K = q (r34 padded to 16), one tile in the layout of a chunk with
// wc = N, PC pieces.
template <int PC>
__global__ void k_split_root(const float* __restrict__ B, int r12, int r34, unsigned char* __restrict__ out) {
  const int n16 = r16(r12), kr16 = r16(r34), ks = kr16 / 16, ng = kr16 / 8;
  const int it = blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= n16 * ng) return;
  const int n = it / ng, kg = it % ng;
  float x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int b = kg * 8 + j;
    x[j] = (n < r12 && b < r34) ? B[(long long)n * r34 + b] : 0.f;
  }
  uint4 pc[PC];
  split8<PC>(x, pc);
  const int off = (kg >> 1) * n16 * 32 + (n >> 3) * 256 + (kg & 1) * 128 + (n & 7) * 16;
#pragma unroll
  for (int q = 0; q < PC; ++q) *reinterpret_cast<uint4*>(out + q * ks * n16 * 32 + off) = pc[q];
}

// stage (128 x r) -> A operand tiles (PC pieces), K padded to r16 with zeros
template <int PC, int NT = TC_THREADS>
__device__ __forceinline__ void stage_to_operand(const float* stage, int r, unsigned char* A) {
  const int ld = stage_ld(r), rb16 = r16(r), ks = rb16 / 16, ng = rb16 / 8;
  for (int it = threadIdx.x; it < TC_TILE * ng; it += NT) {
    const int e = it & (TC_TILE - 1), kg = it >> 7;
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int b = kg * 8 + j;
      x[j] = b < r ? stage[e * ld + b] : 0.f;
    }
    uint4 pc[PC];
    split8<PC>(x, pc);
    const int off = (kg >> 1) * 4096 + (e >> 3) * 256 + (kg & 1) * 128 + (e & 7) * 16;
#pragma unroll
    for (int q = 0; q < PC; ++q) *reinterpret_cast<uint4*>(A + q * ks * 4096 + off) = pc[q];
  }
}

// the thread's own row of the stage into registers (zero beyond r)
__device__ __forceinline__ void stage_to_regs(const float* stage, int r, int e, float* c) {
  const int ld = stage_ld(r);
#pragma unroll
  for (int a = 0; a < 64; ++a) c[a] = a < r ? stage[e * ld + a] : 0.f;
}

// Read-out of one chunk by one warp: the warp takes the half `half` of the chunk's p (NP
// consecutive p, NP x 16 NB <= 64 consecutive columns), loads them with one 64-column
// tensor-memory load and stores c_t[e][p] = sum_a c1[e][a] T[e][(p, a)] into column
// out_col + p.  Columns of p >= p1 (a ragged last chunk) are loaded but not used.
template <int NB>
__device__ __forceinline__ void drain_chunk(const float* creg, uint32_t trow, uint32_t slot_col, int p0, int p1,
                                            int half, int out_col) {
  constexpr int RA16 = 16 * NB;
  constexpr int NP = (tc_w<2>() / RA16) / 2;
  float v[64];
  tmem_ld64(trow + slot_col + (uint32_t)(half * NP * RA16), v);
  tmem_wait_ld();
#pragma unroll
  for (int pi = 0; pi < NP; ++pi) {
    const int p = p0 + half * NP + pi;
    float s4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < RA16; ++a) s4[a & 3] = fmaf(creg[a], v[pi * RA16 + a], s4[a & 3]);
    if (p < p1) tmem_st1(trow + (uint32_t)(out_col + p), (s4[0] + s4[1]) + (s4[2] + s4[3]));
  }
}

// Read-out of one 64-column chunk of the three-piece variant by one warp: the warp loads the
// half `half` of the chunk (32 columns).  RA16 <= 32: its whole p (two of 16 or one of 32) ->
// c_t[e][p] in column out_col + p.  RA16 = 48 or 64: one p per chunk whose a-range spans both
// halves -> the partial sum over the half's a into out_col + p (half 0) or outb_col + p
// (half 1), added at the root.
template <int NB>
__device__ __forceinline__ void drain_chunk3(const float* creg, uint32_t trow, uint32_t slot_col, int p0, int p1,
                                             int half, int out_col, int outb_col) {
  constexpr int RA16 = 16 * NB;
  float v[32];
  tmem_ld32(trow + slot_col + (uint32_t)(half * 32), v);
  tmem_wait_ld();
  if constexpr (RA16 <= 32) {
    constexpr int NP = 32 / RA16;
#pragma unroll
    for (int pi = 0; pi < NP; ++pi) {
      const int p = p0 + half * NP + pi;
      float s4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int a = 0; a < RA16; ++a) s4[a & 3] = fmaf(creg[a], v[pi * RA16 + a], s4[a & 3]);
      if (p < p1) tmem_st1(trow + (uint32_t)(out_col + p), (s4[0] + s4[1]) + (s4[2] + s4[3]));
    }
  } else {
    // RA16 = 48: the second half holds 16 columns of the p; the slot's columns past the chunk
    // are never read (they may hold anything, and 0 x NaN is NaN)
    const int p = p0;
    float s4[4] = {0.f, 0.f, 0.f, 0.f};
    if (half == 0) {
#pragma unroll
      for (int c = 0; c < 32; ++c) s4[c & 3] = fmaf(creg[c], v[c], s4[c & 3]);
    } else {
#pragma unroll
      for (int c = 0; c < RA16 - 32; ++c) s4[c & 3] = fmaf(creg[32 + c], v[c], s4[c & 3]);
    }
    if (p < p1) tmem_st1(trow + (uint32_t)((half ? outb_col : out_col) + p), (s4[0] + s4[1]) + (s4[2] + s4[3]));
  }
}

// Scratch of the prologue, per entry e of a launch (capacity a multiple of TC_TILE):
//   A tiles  tile t = e / 128 at a + t * tc_abytes: the split c2 of node 0 (leaf 1) and of
//            node 1 (leaf 3) in the shared-memory operand layout, copied in one bulk copy;
//   c1       c1[e][node][64] FP32 (leaf 0, leaf 2; zero beyond the rank);
//   rows, w  the entry's stencil rows and weights [4][3] (for the correction epilogue).
template <int PC>
__host__ __device__ __forceinline__ long long tc_abytes(int r1, int r3) {
  return (long long)TC_TILE * (r16(r1) + r16(r3)) * 2 * PC;
}

// Leaf gather of the prologue, a warp per entry row (lanes over the leaf's columns, no
// integer division per item), four rows in flight per warp: row e of c = sum_s w[e][m][s]
// U_m[row_s][:], zero for e >= nT.  Into the stage (row stride stage_ld(r)) for the A
// operands, or into c1[e][node][0..63] (zero beyond r) in global scratch.
constexpr int PRO_THREADS = 256;
template <bool TO_C1>
__device__ __forceinline__ void gather_rows(float* dst, const float* __restrict__ U, int r, int m, int nT,
                                            const int* srow, const float* sw, int node) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ld = stage_ld(r);
  for (int e0 = 4 * warp; e0 < TC_TILE; e0 += 4 * (PRO_THREADS / 32)) {
    const float* u[4][3];
    float w[4][3];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int e = e0 + k;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        u[k][q] = U + (long long)(e < nT ? srow[(e * 4 + m) * 3 + q] : 0) * r;
        w[k][q] = e < nT ? sw[(e * 4 + m) * 3 + q] : 0.f;
      }
    }
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 32) {
      const int col = c0 + lane;
      float v[4][3];
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int q = 0; q < 3; ++q) v[k][q] = col < r ? __ldg(u[k][q] + col) : 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float x = w[k][0] * v[k][0] + w[k][1] * v[k][1] + w[k][2] * v[k][2];
        if (TO_C1) dst[(long long)(e0 + k) * 128 + node * 64 + col] = x;   // zero beyond r (v = 0)
        else if (col < r) dst[(e0 + k) * ld + col] = x;
      }
    }
  }
}

// Prologue of the tensor-core evaluator, one CTA per 128-entry tile: the feet, cells and
// weights, the four leaf gathers, the BF16 split of c2 of both nodes into the A tiles of
// the tile and c1 of both nodes, all into global scratch.  A separate kernel so that these
// latency-bound steps run at several CTAs per SM and overlap one another, while the
// tensor-core kernel (one CTA per SM) starts its MMAs as soon as one bulk copy of the A
// tiles has landed.
template <bool DEV, int PC>
__global__ void __launch_bounds__(PRO_THREADS)
k_tc_prologue(GridDesc g, HTView<float> ht_arg, const EvalParams<float>* __restrict__ P, EvalArgs a,
              TcScratch sc) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  HTView<float> ht;
  if (DEV) {
    const EvalParams<float> q = *P;
    ht = q.ht;
    a.tau = q.tau;
    a.E = q.E;
    a.E32 = q.E32;
    a.foot_euler = q.foot_euler;
  } else {
    ht = ht_arg;
  }
  if ((a.done && *a.done) || (a.skip && *a.skip)) return;
  if (a.kidx) a.pivot += *a.kidx;
  const long long e0 = (long long)blockIdx.x * TC_TILE;
  const long long n_act = a.nact ? min(a.n, (long long)(*a.nact) * a.nper) : a.n;
  if (e0 >= n_act) return;
  const int nT = (int)min((long long)TC_TILE, n_act - e0);
  const int tid = threadIdx.x;
  float* sw = reinterpret_cast<float*>(smem_raw);                     // 128 x 12
  int* srow = reinterpret_cast<int*>(sw + TC_TILE * 12);              // 128 x 12
  float* stage = reinterpret_cast<float*>(smem_raw + PRO_HEAD_BYTES);
  if (tid < nT) {
    int idx[4];
    decode_tuple(g, a, e0 + tid, idx);
    float foot[4];
    int r[12];
    float w[12];
    foot_cells_ft<2>(g, a.E32, a.E, a.tau, a.foot_euler, idx, foot, r, w);   // d = 4: two spatial dimensions
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      srow[tid * 12 + k] = r[k];
      sw[tid * 12 + k] = w[k];
      sc.rows[(e0 + tid) * 12 + k] = r[k];
      sc.w[(e0 + tid) * 12 + k] = w[k];
    }
  }
  __syncthreads();
  unsigned char* At = sc.a + (long long)blockIdx.x * tc_abytes<PC>(ht.r[1], ht.r[3]);
  float* c1 = sc.c1 + e0 * 128;
  // c1 of both nodes straight to the scratch, then c2 of each node through the stage
  gather_rows<true>(c1, ht.U[0], ht.r[0], 0, nT, srow, sw, 0);
  gather_rows<true>(c1, ht.U[2], ht.r[2], 2, nT, srow, sw, 1);
  gather_rows<false>(stage, ht.U[1], ht.r[1], 1, nT, srow, sw, 0);
  __syncthreads();
  stage_to_operand<PC, PRO_THREADS>(stage, ht.r[1], At);
  __syncthreads();
  gather_rows<false>(stage, ht.U[3], ht.r[3], 3, nT, srow, sw, 0);
  __syncthreads();
  stage_to_operand<PC, PRO_THREADS>(stage, ht.r[3], At + (long long)TC_TILE * r16(ht.r[1]) * 2 * PC);
}

size_t tc_prologue_smem(const int* r6) {
  int rmax = 1;
  for (int m = 0; m < 4; ++m) rmax = r6[m] > rmax ? r6[m] : rmax;
  return (size_t)PRO_HEAD_BYTES + (size_t)4 * TC_TILE * stage_ld(rmax);
}

template <bool DEV, int PC>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_sl_eval_tc(GridDesc g, HTView<float> ht_arg, CorrView corr_arg, const EvalParams<float>* __restrict__ P,
             EvalArgs a, const unsigned char* __restrict__ b12, const unsigned char* __restrict__ b34, int* err,
             TcScratch sc, const unsigned char* __restrict__ broot) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // full, mma_done, drained (per stage); A tiles; root B; root MMAs
  __shared__ __align__(8) unsigned long long s_bar[3 * TC_STAGES + 3];
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  HTView<float> ht;
  CorrView corr;
  if (DEV) {
    const EvalParams<float> q = *P;
    ht = q.ht;
    corr = q.corr;
    a.tau = q.tau;
    a.E = q.E;
    a.E32 = q.E32;
    a.foot_euler = q.foot_euler;
  } else {
    ht = ht_arg;
    corr = corr_arg;
  }
  if ((a.done && *a.done) || (a.skip && *a.skip)) return;
  if (a.kidx) {
    const int kk = *a.kidx;
    a.pivot += kk;
    a.kterms = kk;
    a.out += kk * a.out_stride;
  }
  const long long e0 = (long long)blockIdx.x * TC_TILE;
  // a block of fibres evaluates only its *nact active fibres
  const long long n_act = a.nact ? min(a.n, (long long)(*a.nact) * a.nper) : a.n;
  if (e0 >= n_act) return;
  const int nT = (int)min((long long)TC_TILE, n_act - e0);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const TcLayout L = tc_layout<PC>(ht.r[0], ht.r[1], ht.r[2], ht.r[3], ht.r12, ht.r34);
  double* sval = reinterpret_cast<double*>(smem_raw);                // 128
  float* spart = reinterpret_cast<float*>(sval + TC_TILE);            // 128
  unsigned char* A0 = smem_raw + L.A0;
  unsigned char* A1 = smem_raw + L.A1;
  const uint32_t bslot = smem_u32(smem_raw + L.B);
  const uint32_t full = smem_u32(&s_bar[0]), mdone = smem_u32(&s_bar[TC_STAGES]),
                 drained = smem_u32(&s_bar[2 * TC_STAGES]), abar = smem_u32(&s_bar[3 * TC_STAGES]),
                 rbar = smem_u32(&s_bar[3 * TC_STAGES + 1]), rdone = smem_u32(&s_bar[3 * TC_STAGES + 2]);
  const long long abytes = tc_abytes<PC>(ht.r[1], ht.r[3]);

  const TcNode N0 = tc_node<PC>(ht.r[0], ht.r[1], ht.r12, smem_u32(A0), b12, tc_out12<PC>());
  const TcNode N1 = tc_node<PC>(ht.r[2], ht.r[3], ht.r34, smem_u32(A1), b34, tc_out34<PC>());
  const int nchunk = N0.nch + N1.nch;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < TC_STAGES; ++i) {
      mbar_init(full + 8 * i, 1);
      mbar_init(mdone + 8 * i, 1);
      mbar_init(drained + 8 * i, TC_CONSUMERS / 32);
    }
    mbar_init(abar, 1);
    mbar_init(rbar, 1);
    mbar_init(rdone, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s_tmem;

  // chunk j of the column stream: its node (by value: field selects, no local memory),
  // local chunk index and width
  auto chunk = [&](int j, TcNode& N, int& cl, int& wc) {
    const bool first = j < N0.nch;
    N = first ? N0 : N1;
    cl = first ? j : j - N0.nch;
    wc = min(N.w, N.ntot - cl * N.w);
  };
  auto issue_copy = [&](int j) {
    TcNode N;
    int cl, wc;
    chunk(j, N, cl, wc);
    const uint32_t bytes = (uint32_t)(wc * N.rb16 * 2 * PC);
    const int s = j % TC_STAGES;
    mbar_expect_tx(full + 8 * s, bytes);
    bulk_g2s(bslot + s * L.slot, N.bg + (long long)cl * N.w * N.rb16 * 2 * PC, bytes, full + 8 * s);
  };
  const bool copier = tid == TC_COPY_WARP * 32, issuer = tid == TC_MMA_WARP * 32;
  int n_copy = 0;
  if (copier) {
    // the tile's A operands (both nodes, written by the prologue) in one bulk copy
    mbar_expect_tx(abar, (uint32_t)abytes);
    bulk_g2s(smem_u32(A0), sc.a + (long long)blockIdx.x * abytes, (uint32_t)abytes, abar);
    for (; n_copy < TC_STAGES && n_copy < nchunk; ++n_copy) issue_copy(n_copy);
  }

  // 2. c1 of node 0 into registers (from the prologue's scratch; zero beyond the rank)
  const int e_own = 32 * (warp & 3) + lane;   // the tensor-memory lane this warp may access
  const int half = (warp >> 2) & 1;           // the two warps of a lane quadrant split the p's
  const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  float creg[64];
  auto load_c1 = [&](int node) {
    const float4* src = reinterpret_cast<const float4*>(sc.c1 + (e0 + e_own) * 128 + node * 64);
#pragma unroll
    for (int q4 = 0; q4 < 16; ++q4) {
      const float4 v = src[q4];
      creg[4 * q4] = v.x;
      creg[4 * q4 + 1] = v.y;
      creg[4 * q4 + 2] = v.z;
      creg[4 * q4 + 3] = v.w;
    }
  };
  if (warp < 8) load_c1(0);

  // 3. the chunk stream
  int n_mma = 0;
  if (issuer) {
    if (!wait_one(abar, 0)) {
      *(volatile int*)&s_abort = 1;
      atomicExch(err, 1);
    }
    for (int j = 0; j < nchunk; ++j) {
      if (*(volatile int*)&s_abort) break;
      const int s = j % TC_STAGES;
      bool ok = wait_one(full + 8 * s, (j / TC_STAGES) & 1);
      if (ok && j >= TC_STAGES) ok = wait_one(drained + 8 * s, ((j - TC_STAGES) / TC_STAGES) & 1);
      if (!ok) {
        *(volatile int*)&s_abort = 1;
        atomicExch(err, 1);
        break;
      }
      TcNode N;
      int cl, wc;
      chunk(j, N, cl, wc);
      fence_after();
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(wc >> 3) << 17) |
                             ((uint32_t)(TC_TILE >> 4) << 24);
      const uint32_t dt = tmem + (uint32_t)(s * tc_w<PC>());
      const uint32_t bb = bslot + s * L.slot;
      for (int k = 0; k < N.ks; ++k) {
        // piece q of the A / B operands at K-step k
        auto ad = [&](int q) { return tc_desc(N.a_addr + (q * N.ks + k) * 4096); };
        auto bd = [&](int q) { return tc_desc(bb + (q * N.ks + k) * wc * 32); };
        mma_bf16(dt, ad(0), bd(0), idesc, k > 0 ? 1u : 0u);
        mma_bf16(dt, ad(0), bd(1), idesc, 1u);
        mma_bf16(dt, ad(1), bd(0), idesc, 1u);
        if constexpr (PC == 3) {
          mma_bf16(dt, ad(0), bd(2), idesc, 1u);
          mma_bf16(dt, ad(2), bd(0), idesc, 1u);
          mma_bf16(dt, ad(1), bd(1), idesc, 1u);
        }
      }
      mma_commit(mdone + 8 * s);
      n_mma = j + 1;
    }
  } else if (copier) {
    for (int j = TC_STAGES; j < nchunk; ++j) {
      if (*(volatile int*)&s_abort) break;
      const int s = j % TC_STAGES;
      if (!wait_one(mdone + 8 * s, ((j - TC_STAGES) / TC_STAGES) & 1)) {
        *(volatile int*)&s_abort = 1;
        atomicExch(err, 1);
        break;
      }
      issue_copy(j);
      n_copy = j + 1;
    }
  } else if (warp < 8) {
    for (int c = 0; c < nchunk; ++c) {
      if (c == N0.nch) load_c1(1);   // node switch: c1 of node 1
      const int s = c % TC_STAGES;
      if (!__any_sync(0xffffffffu, *(volatile int*)&s_abort != 0)) {
        if (!wait_warp(mdone + 8 * s, (c / TC_STAGES) & 1)) {
          if (lane == 0) {
            *(volatile int*)&s_abort = 1;
            atomicExch(err, 1);
          }
        } else {
          fence_after();
          TcNode N;
          int cl, wc;
          chunk(c, N, cl, wc);
          const int p0 = cl * N.pc, p1 = min(N.rp, p0 + N.pc);
          const uint32_t sc = (uint32_t)(s * tc_w<PC>());
          if constexpr (PC == 2) {
            switch (N.ra16) {
              case 16: drain_chunk<1>(creg, trow, sc, p0, p1, half, N.out_col); break;
              case 32: drain_chunk<2>(creg, trow, sc, p0, p1, half, N.out_col); break;
              case 48: drain_chunk<3>(creg, trow, sc, p0, p1, half, N.out_col); break;
              default: drain_chunk<4>(creg, trow, sc, p0, p1, half, N.out_col); break;
            }
          } else {
            const int outb = N.out_col == tc_out12<PC>() ? tc_out12b<PC>() : tc_out34b<PC>();
            switch (N.ra16) {
              case 16: drain_chunk3<1>(creg, trow, sc, p0, p1, half, N.out_col, outb); break;
              case 32: drain_chunk3<2>(creg, trow, sc, p0, p1, half, N.out_col, outb); break;
              case 48: drain_chunk3<3>(creg, trow, sc, p0, p1, half, N.out_col, outb); break;
              default: drain_chunk3<4>(creg, trow, sc, p0, p1, half, N.out_col, outb); break;
            }
          }
          fence_before();
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(drained + 8 * s);
    }
  }

  // copies and MMAs still in flight (only after an abort) end before the CTA does
  if (copier) wait_one(abar, 0);
  if (copier)
    for (int k = n_copy - TC_STAGES < 0 ? 0 : n_copy - TC_STAGES; k < n_copy; ++k)
      wait_one(full + 8 * (k % TC_STAGES), (k / TC_STAGES) & 1);
  if (issuer && n_mma > 0) wait_one(mdone + 8 * ((n_mma - 1) % TC_STAGES), ((n_mma - 1) / TC_STAGES) & 1);
  __syncwarp();
  tmem_wait_st();
  fence_before();
  __syncthreads();
  fence_after();
  const bool ok = *(volatile int*)&s_abort == 0;

  if (ok) {
    // 4. root on the tensor cores: T[e][p] = sum_q c34[e][q] Broot[p][q], a [128 x r34] x
    //    [r34 x r12] GEMM (c34 split into PC BF16 pieces as the A operand over the freed A
    //    region, the pre-split Broot bulk-copied after it), then sum_p c12[e][p] T[e][p] per
    //    entry; the two warps of a lane quadrant take p < 32 and p >= 32
    const int rl = ht.r12, rr = ht.r34;
    const int n16 = r16(rl), kr16 = r16(rr), ksr = kr16 / 16;
    unsigned char* RA = smem_raw + L.A0;
    const uint32_t rb_addr = smem_u32(smem_raw + L.rootB);
    const uint32_t rbytes = (uint32_t)(n16 * kr16 * 2 * PC);
    bool root_mma = false;
    if (copier) {
      mbar_expect_tx(rbar, rbytes);
      bulk_g2s(rb_addr, broot, rbytes, rbar);
    }
    float c12h[32];
    if (warp < 8) {
      float c34[64];
      tmem_ld64(trow + tc_out34<PC>(), c34);
      tmem_ld32(trow + tc_out12<PC>() + half * 32, c12h);
      tmem_wait_ld();
      if constexpr (PC == 3) {
        // the second partial sums of nodes whose a-range spans both halves of a chunk, 16
        // columns at a time
        float cb[16];
        if (N1.ra16 > 32) {
#pragma unroll
          for (int q0 = 0; q0 < 64; q0 += 16) {
            tmem_ld16(trow + tc_out34b<PC>() + q0, cb);
            tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 16; ++q) c34[q0 + q] += cb[q];
          }
        }
        if (N0.ra16 > 32) {
#pragma unroll
          for (int q0 = 0; q0 < 32; q0 += 16) {
            tmem_ld16(trow + tc_out12b<PC>() + half * 32 + q0, cb);
            tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 16; ++q) c12h[q0 + q] += cb[q];
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 64; ++q)
        if (q >= rr) c34[q] = 0.f;
      // row e_own of the A operand: this warp's half of the 8-column K groups
#pragma unroll
      for (int g4 = 0; g4 < 4; ++g4) {
        const int kg = half * 4 + g4;
        if (kg * 8 < kr16) {
          float x[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) x[j] = c34[kg * 8 + j];
          uint4 pcs[PC];
          split8<PC>(x, pcs);
          const int off = (kg >> 1) * 4096 + (e_own >> 3) * 256 + (kg & 1) * 128 + (e_own & 7) * 16;
#pragma unroll
          for (int q = 0; q < PC; ++q) *reinterpret_cast<uint4*>(RA + q * ksr * 4096 + off) = pcs[q];
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // A operand -> tensor cores
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (issuer) {
      if (wait_one(rbar, 0)) {
        root_mma = true;
        fence_after();
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n16 >> 3) << 17) |
                               ((uint32_t)(TC_TILE >> 4) << 24);
        for (int k = 0; k < ksr; ++k) {
          auto ad = [&](int q) { return tc_desc(smem_u32(RA) + (q * ksr + k) * 4096); };
          auto bd = [&](int q) { return tc_desc(rb_addr + (q * ksr + k) * n16 * 32); };
          mma_bf16(tmem, ad(0), bd(0), idesc, k > 0 ? 1u : 0u);
          mma_bf16(tmem, ad(0), bd(1), idesc, 1u);
          mma_bf16(tmem, ad(1), bd(0), idesc, 1u);
          if constexpr (PC == 3) {
            mma_bf16(tmem, ad(0), bd(2), idesc, 1u);
            mma_bf16(tmem, ad(2), bd(0), idesc, 1u);
            mma_bf16(tmem, ad(1), bd(1), idesc, 1u);
          }
        }
        mma_commit(rdone);
      } else {
        *(volatile int*)&s_abort = 1;
        atomicExch(err, 1);
      }
    }
    if (warp < 8) {
      float acc = 0.f;
      if (wait_warp(rdone, 0)) {
        fence_after();
        float t[32];
        tmem_ld32(trow + (uint32_t)(half * 32), t);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (half * 32 + i < rl) acc = fmaf(c12h[i], t[i], acc);
      } else if (lane == 0) {
        *(volatile int*)&s_abort = 1;
        atomicExch(err, 1);
      }
      if (half == 1) spart[e_own] = acc;
      consumer_sync();
      if (half == 0) sval[e_own] = (double)(acc + spart[e_own]);
    }
    // the root's copy and MMAs have completed before the CTA leaves (waits bounded)
    if (copier) wait_one(rbar, 0);
    if (issuer && root_mma) wait_one(rdone, 0);
    __syncthreads();
    // 5. correction and residual epilogue
    if (tid < nT) {
      double val = sval[tid];
      if (corr.has) val += (double)correction_rw_ft<2>(g, corr, sc.rows + (e0 + tid) * 12, sc.w + (e0 + tid) * 12);
      const long long e = e0 + tid;
      if (a.X) {
        const long long fib = a.nper ? e / a.nper : 0;
        const long long piv = (long long)a.pivot[fib];
        const long long ey = a.nper ? e - fib * a.nper : e;
        for (int l = 0; l < a.kterms; ++l) val -= a.X[piv + l * a.ldX] * a.Y[ey + l * a.ldY];
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

// The bounded-wait path of the evaluator exercised on its own: one thread waits for the first
// phase of an mbarrier that nothing arrives on, gives up after `polls` polls and records it
// in *status (1: gave up, 0: the phase completed).
__global__ void k_wait_probe(long long polls, int* status) {
  __shared__ __align__(8) unsigned long long bar;
  const uint32_t b = smem_u32(&bar);
  if (threadIdx.x == 0) {
    mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) *status = wait_one_n(b, 0, polls) ? 0 : 1;
}

}  // namespace

size_t sl_eval_tc_smem(const int* r6, int pieces) {
  return (size_t)(pieces == 3 ? tc_layout<3>(r6[0], r6[1], r6[2], r6[3], r6[4], r6[5]).total
                              : tc_layout<2>(r6[0], r6[1], r6[2], r6[3], r6[4], r6[5]).total);
}

long long tc_split_bytes(int pieces) { return 64LL * 64 * 64 * 2 * pieces; }

long long tc_scratch_bytes(long long cap) {
  // A tiles (at most 128 + 128 padded columns x 3 BF16 pieces per entry), c1 (2 x 64 FP32),
  // rows and weights (12 + 12)
  return cap * ((128 + 128) * 2 * 3 + 128 * 4 + 24 * 4);
}

TcScratch tc_scratch_view(void* base, long long cap) {
  TcScratch sc;
  unsigned char* p = static_cast<unsigned char*>(base);
  sc.a = p;
  p += cap * (128 + 128) * 2 * 3;
  sc.c1 = reinterpret_cast<float*>(p);
  p += cap * 128 * 4;
  sc.rows = reinterpret_cast<int*>(p);
  p += cap * 12 * 4;
  sc.w = reinterpret_cast<float*>(p);
  sc.cap = cap;
  return sc;
}

cudaError_t sl_eval_tc_init_attrs() {
  const int mx = 220 * 1024;
  const int mp = (int)(PRO_HEAD_BYTES + 4 * TC_TILE * stage_ld(64));
  cudaError_t e = cudaFuncSetAttribute(k_tc_prologue<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mp);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tc_prologue<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mp);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tc_prologue<true, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, mp);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tc_prologue<false, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, mp);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sl_eval_tc<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sl_eval_tc<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sl_eval_tc<true, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sl_eval_tc<false, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  return e;
}

cudaError_t split_root_bf16(const float* Broot, int r12, int r34, void* out, int pieces, cudaStream_t s) {
  if (r12 < 1 || r34 < 1 || r12 > 64 || r34 > 64 || (pieces != 2 && pieces != 3)) return cudaErrorInvalidValue;
  const int n = r16(r12) * (r16(r34) / 8);
  if (pieces == 3)
    slar::count_launch(), k_split_root<3><<<(n + 255) / 256, 256, 0, s>>>(Broot, r12, r34,
                                                                         static_cast<unsigned char*>(out));
  else
    slar::count_launch(), k_split_root<2><<<(n + 255) / 256, 256, 0, s>>>(Broot, r12, r34,
                                                                         static_cast<unsigned char*>(out));
  return cudaGetLastError();
}

cudaError_t split_transfer_bf16(const float* B, int rp, int ra, int rb, void* out, int pieces, cudaStream_t s) {
  if (rp < 1 || ra < 1 || rb < 1 || rp > 64 || ra > 64 || rb > 64 || (pieces != 2 && pieces != 3))
    return cudaErrorInvalidValue;
  const long long n = (long long)rp * r16(ra) * (r16(rb) / 8);
  if (pieces == 3)
    slar::count_launch(), k_split_bf16<3><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(B, rp, ra, rb,
                                                                                      static_cast<unsigned char*>(out));
  else
    slar::count_launch(), k_split_bf16<2><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(B, rp, ra, rb,
                                                                                      static_cast<unsigned char*>(out));
  return cudaGetLastError();
}

cudaError_t launch_sl_eval_tc(const GridDesc& g, const HTView<float>& ht, const CorrView& corr, const EvalArgs& a0,
                              const void* b12, const void* b34, const void* broot_, int* err, int pieces,
                              const TcScratch& sc, cudaStream_t s) {
  const unsigned char* broot = static_cast<const unsigned char*>(broot_);
  if (a0.n <= 0) return cudaSuccess;
  if (g.d != 4 || sc.cap < TC_TILE) return cudaErrorInvalidValue;
  // entries beyond the scratch capacity: index tuples are evaluated in chunks of it
  if (a0.n > sc.cap && (a0.mode != EVAL_TUPLES || a0.X)) return cudaErrorInvalidValue;
  const int r6[6] = {ht.r[0], ht.r[1], ht.r[2], ht.r[3], ht.r12, ht.r34};
  const size_t sm = sl_eval_tc_smem(r6, pieces);
  const size_t smp = tc_prologue_smem(r6);
  const unsigned char* p12 = static_cast<const unsigned char*>(b12);
  const unsigned char* p34 = static_cast<const unsigned char*>(b34);
  for (long long off = 0; off < a0.n; off += sc.cap) {
    EvalArgs a = a0;
    if (a0.n > sc.cap) {
      a.n = a0.n - off < sc.cap ? a0.n - off : sc.cap;
      a.idx = a0.idx + off * g.d;
      a.out = a0.out + off;
    }
    const long long blocks = (a.n + TC_TILE - 1) / TC_TILE;
    if (pieces == 3) {
      slar::count_launch(), k_tc_prologue<false, 3><<<(unsigned)blocks, PRO_THREADS, smp, s>>>(g, ht, nullptr, a, sc);
      slar::count_launch(), k_sl_eval_tc<false, 3><<<(unsigned)blocks, TC_THREADS, sm, s>>>(g, ht, corr, nullptr, a,
                                                                                           p12, p34, err, sc, broot);
    } else {
      slar::count_launch(), k_tc_prologue<false, 2><<<(unsigned)blocks, PRO_THREADS, smp, s>>>(g, ht, nullptr, a, sc);
      slar::count_launch(), k_sl_eval_tc<false, 2><<<(unsigned)blocks, TC_THREADS, sm, s>>>(g, ht, corr, nullptr, a,
                                                                                           p12, p34, err, sc, broot);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_sl_eval_tc_dev(const GridDesc& g, const EvalParams<float>* P, const EvalArgs& a, const void* b12,
                                  const void* b34, const void* broot_, int* err, int pieces, size_t sm,
                                  const TcScratch& sc, cudaStream_t s) {
  const unsigned char* broot = static_cast<const unsigned char*>(broot_);
  if (g.d != 4 || a.n > sc.cap) return cudaErrorInvalidValue;
  const long long blocks = (a.n + TC_TILE - 1) / TC_TILE;
  const unsigned char* p12 = static_cast<const unsigned char*>(b12);
  const unsigned char* p34 = static_cast<const unsigned char*>(b34);
  // the prologue's shared memory for the largest ranks (the ranks are read on the device)
  const size_t smp = (size_t)PRO_HEAD_BYTES + (size_t)4 * TC_TILE * stage_ld(64);
  if (pieces == 3) {
    slar::count_launch(), k_tc_prologue<true, 3><<<(unsigned)blocks, PRO_THREADS, smp, s>>>(g, HTView<float>{}, P, a,
                                                                                         sc);
    slar::count_launch(), k_sl_eval_tc<true, 3><<<(unsigned)blocks, TC_THREADS, sm, s>>>(
        g, HTView<float>{}, CorrView{}, P, a, p12, p34, err, sc, broot);
  } else {
    slar::count_launch(), k_tc_prologue<true, 2><<<(unsigned)blocks, PRO_THREADS, smp, s>>>(g, HTView<float>{}, P, a,
                                                                                         sc);
    slar::count_launch(), k_sl_eval_tc<true, 2><<<(unsigned)blocks, TC_THREADS, sm, s>>>(
        g, HTView<float>{}, CorrView{}, P, a, p12, p34, err, sc, broot);
  }
  return cudaGetLastError();
}

}  // namespace slar

extern "C" slar_status slar_wait_probe(long long polls, int* status_dev, void* stream) {
  if (polls < 1 || polls > slar::TC_WAIT_LIMIT || !status_dev) return SLAR_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  slar::count_launch(), slar::k_wait_probe<<<1, 32, 0, s>>>(polls, status_dev);
  if (cudaGetLastError() != cudaSuccess) return SLAR_ECUDA;
  int h = 0;
  if (cudaMemcpyAsync(&h, status_dev, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SLAR_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SLAR_ECUDA;
  return h ? SLAR_ETIMEOUT : SLAR_OK;
}
