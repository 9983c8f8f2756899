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
// through a shared-memory ring of B tiles (4 slots for BF16x3, 3 for BF16x6) and a 3-slot
// tensor-memory ring of results:
//   warp 9 (one thread)   bulk-copies chunk j's pre-split B tile (all pieces) into shared
//                         slot j mod S once the MMAs of chunk j - S have released it,
//   warps 8 and 10        (one thread each, the even and the odd chunks) issue chunk j's
//                         3 (6) x K/16 MMAs into tensor-memory slot j % 3 once the tile has
//                         landed and chunk j - 3 has been read out, and commit them to two
//                         mbarriers (result ready, shared slot free).  A thread's MMA issue
//                         stalls while the tensor pipe executes the MMAs before it, so one
//                         issuer would leave the pipe idle during its own waits; with two,
//                         one issues while the other waits,
//   warps 0-7             read chunk j out of tensor memory (one load of W/2 columns per
//                         warp: the warp pair of a lane quadrant splits the chunk's columns
//                         in halves), dot them with c1 held in registers and store c_t[e][p]
//                         in shared memory; each warp then arrives on the slot's mbarrier.
//                         A BF16x6 p split across the two halves leaves two partial sums,
//                         added before the root contraction.
// The MMA's A operand, c2 of both nodes split into BF16 pieces, sits in tensor memory
// (written once per CTA by warps 0-7 from the prologue's rows), and only the B tiles are read
// from shared memory: two threads issuing m128n128k16 MMAs back to back measured ~87 cycles
// per MMA with both operands in shared memory and ~70 with A in tensor memory (ideal 64).
// c1 of the current node sits in registers (the thread's own entry); c_12 and c_34 stay in
// shared memory for the root contraction (c34 x Broot on the tensor cores, A = c34 in tensor
// memory) and the correction / residual epilogue of the SIMT evaluator.
// Shared-memory B layout (canonical, no swizzle, K-major): K-step s | 8-row group | K core
// matrix | 8 rows x 16 bytes; byte (row, kk) = (row / 8) 256 + (kk / 8) 128 + (row % 8) 16 +
// (kk % 8) 2 for kk < 16, i.e. leading (K) byte offset 128, stride (N) byte offset 256.
// Tensor-memory A layout: lane = row, column = 32-bit word holding two K-elements (the first
// in the low half); piece q, K-step k at columns (q ks + k) 8 .. + 7 from the node's base.
// Every wait is bounded: a wait that runs out sets *err, the CTA skips the remaining work,
// waits (bounded) for its copies and MMAs in flight and frees its tensor memory.
#include <cuda_bf16.h>

#include "common.cuh"
#include "eval_device.cuh"

namespace slar {
namespace {

constexpr int TC_TILE = 128;
constexpr int TC_CONSUMERS = 256;        // warps 0-7
constexpr int TC_MMA_WARP = 8;           // issues the even chunks
constexpr int TC_COPY_WARP = 9;
constexpr int TC_MMA2_WARP = 10;         // issues the odd chunks
constexpr int TC_THREADS = 352;
constexpr int TC_STAGES = 3;             // tensor-memory result slots
constexpr int TC_TMEM_COLS = 512;        // 3 chunk slots and the A operands of both nodes

// Operands split into PC BF16 pieces: PC = 2 (x = hi + lo, three products hh + hl + lh, about
// 2^-16 relative per product) or PC = 3 (x = x1 + x2 + x3, six products 11 + 12 + 21 + 13 + 31
// + 22, about 2^-24).  Columns per chunk: 128 with two pieces; 64 with three, so that the
// ring of 1.5x larger B slots fits in shared memory beside the results at rank 64.
// Tensor-memory columns: three chunk slots, then the A operands of node 0 and node 1 (PC x 32
// columns each at rank 64).  With three pieces the read-out of a p whose a-range spans both
// 32-column halves of a chunk leaves two partial sums (the second in a second result array).
template <int PC> __host__ __device__ constexpr int tc_w() { return PC == 2 ? 128 : 64; }
template <int PC> __host__ __device__ constexpr int tc_sstages() { return PC == 2 ? 4 : 3; }
template <int PC> __host__ __device__ constexpr int tc_acol(int node) { return 3 * tc_w<PC>() + node * 32 * PC; }
constexpr long long TC_WAIT_LIMIT = 1LL << 22;
constexpr int TC_HEAD_BYTES = 2048;      // values and partial sums of the root
constexpr int PRO_SMEM_BYTES = 128 * 12 * 8;   // prologue: stencil rows and weights of up to 128 entries
constexpr int TC_MIN_SMEM = 120 * 1024;  // one CTA per SM: the 512-column allocation never waits

__host__ __device__ __forceinline__ int r16(int r) { return ((r + 15) / 16) * 16; }
template <int PC>
__host__ __device__ __forceinline__ int tc_width(int ra16) { return (tc_w<PC>() / ra16) * ra16; }

struct TcLayout {
  int out, outb, B, slot, total;
};
constexpr int TC_OUT_BYTES = 2 * 64 * TC_TILE * 4;   // c_t[node][p][e], FP32

template <int PC>
__host__ __device__ __forceinline__ TcLayout tc_layout(int r0, int r1, int r2, int r3, int r12, int r34) {
  TcLayout L;
  int o = TC_HEAD_BYTES;
  L.out = o; o += TC_OUT_BYTES;
  L.outb = L.out;
  if (PC == 3) { L.outb = o; o += TC_OUT_BYTES; }
  const int s0 = tc_width<PC>(r16(r0)) * r16(r1) * 2 * PC, s1 = tc_width<PC>(r16(r2)) * r16(r3) * 2 * PC;
  L.slot = s0 > s1 ? s0 : s1;
  L.B = o; o += tc_sstages<PC>() * L.slot;
  // the pre-split Broot of the root contraction reuses the B ring once the stream is over
  const int root_end = L.B + r16(r12) * r16(r34) * 2 * PC;
  if (root_end > o) o = root_end;
  L.total = o > TC_MIN_SMEM ? o : TC_MIN_SMEM;
  return L;
}

// one transfer node as the chunk stream sees it
struct TcNode {
  int ra, rp, ra16, rb16, ks, w, pc, ntot, nch;
  int out_off;                     // c_t of the node in the shared result arrays
  uint32_t a_col;                  // A operand (c2 split): tensor-memory column
  const unsigned char* bg;         // pre-split B tiles in global memory
};

template <int PC>
__device__ __forceinline__ TcNode tc_node(int ra, int rb, int rp, uint32_t a_col, const unsigned char* bg,
                                          int out_off) {
  TcNode n;
  n.ra = ra; n.rp = rp;
  n.ra16 = r16(ra); n.rb16 = r16(rb); n.ks = n.rb16 / 16;
  n.w = tc_width<PC>(n.ra16); n.pc = n.w / n.ra16;
  n.ntot = rp * n.ra16; n.nch = (n.ntot + n.w - 1) / n.w;
  n.out_off = out_off;
  n.a_col = a_col;
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

// A from tensor memory (address a_tmem), B from shared memory (descriptor)
template <int ACC>
__device__ __forceinline__ void mma_bf16c(uint32_t tmem_d, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n"
      ::"r"(tmem_d), "r"(a_tmem), "l"(bdesc), "r"(idesc), "n"(ACC)
      : "memory");
}

// The MMAs of one chunk: KS K-steps x the split's products.  a0 is the tensor-memory address
// of piece 0 at K-step 0 (K-step stride 8 columns, piece stride KS x 8); b0 the descriptor of
// piece 0 at K-step 0, whose start-address field holds the byte address / 16 (all shared
// addresses stay below 2^18, so the field does not overflow), hence the descriptor of a
// block at byte offset o is b0 + o / 16: K-step stride wc x 32 bytes (bk = wc x 2), piece
// stride KS x wc x 32.
template <int PC, int KS>
__device__ __forceinline__ void issue_chunk(uint32_t dt, uint32_t a0, uint64_t b0, uint32_t bk, uint32_t idesc) {
  constexpr uint32_t AQ = KS * 8;
  const uint32_t BQ = KS * bk;
#pragma unroll
  for (int k = 0; k < KS; ++k) {
    const uint32_t a = a0 + k * 8;
    const uint64_t b = b0 + k * bk;
    if (k == 0)
      mma_bf16c<0>(dt, a, b, idesc);
    else
      mma_bf16c<1>(dt, a, b, idesc);
    mma_bf16c<1>(dt, a, b + BQ, idesc);
    mma_bf16c<1>(dt, a + AQ, b, idesc);
    if constexpr (PC == 3) {
      mma_bf16c<1>(dt, a, b + 2 * BQ, idesc);
      mma_bf16c<1>(dt, a + 2 * AQ, b, idesc);
      mma_bf16c<1>(dt, a + AQ, b + BQ, idesc);
    }
  }
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

// bounded wait of a whole warp: lane 0 polls (one request per poll instead of 32), then
// every lane observes the completed phase itself (its own acquire); true on every lane
__device__ __forceinline__ bool wait_warp(uint32_t bar, uint32_t parity) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = wait_one(bar, parity) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (!ok) return false;
  return __all_sync(0xffffffffu, mbar_try_wait(bar, parity) || wait_one(bar, parity));
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
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint4 v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w)
               : "memory");
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

// Read-out of one chunk by one warp: the warp takes the half `half` of the chunk's p (NP
// consecutive p, NP x 16 NB <= 64 consecutive columns), loads them with one 64-column
// tensor-memory load and stores c_t[e][p] = sum_a c1[e][a] T[e][(p, a)] at so[p x 128] (so:
// the node's result array at the thread's entry).  Columns of p >= p1 (a ragged last chunk)
// are loaded but not used.
template <int NB>
__device__ __forceinline__ void drain_chunk(const float* creg, uint32_t trow, uint32_t slot_col, int p0, int p1,
                                            int half, float* so) {
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
    if (p < p1) so[p * TC_TILE] = (s4[0] + s4[1]) + (s4[2] + s4[3]);
  }
}

// Read-out of one 64-column chunk of the three-piece variant by one warp: the warp loads the
// half `half` of the chunk (32 columns).  RA16 <= 32: its whole p (two of 16 or one of 32) ->
// c_t[e][p] at so[p x 128].  RA16 = 48 or 64: one p per chunk whose a-range spans both halves
// -> the partial sum over the half's a at so[p x 128] (half 0) or sob[p x 128] (half 1), added
// at the root.
template <int NB>
__device__ __forceinline__ void drain_chunk3(const float* creg, uint32_t trow, uint32_t slot_col, int p0, int p1,
                                             int half, float* so, float* sob) {
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
      if (p < p1) so[p * TC_TILE] = (s4[0] + s4[1]) + (s4[2] + s4[3]);
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
    if (p < p1) (half ? sob : so)[p * TC_TILE] = (s4[0] + s4[1]) + (s4[2] + s4[3]);
  }
}

// Scratch of the prologue, per entry e of a launch (capacity a multiple of TC_TILE):
//   A rows   tile t = e / 128 at a + t * tc_abytes: the split c2 of node 0 (leaf 1) and of
//            node 1 (leaf 3) as the rows of the tensor-memory A operand: the PC BF16 pieces
//            of row e, two K-elements per 32-bit word in the tensor-memory order (piece q,
//            K-step k, word w: elements 16k + 2w and 16k + 2w + 1), as 16-byte groups g
//            (words 4g .. 4g + 3) at (g x 128 + e) x 16 bytes, so that a warp's 32 rows load
//            coalesced; K padded to r16 with zeros;
//   c1       c1[e][node][64] FP32 (leaf 0, leaf 2; zero beyond the rank);
//   rows, w  the entry's stencil rows and weights [4][3] (for the correction epilogue).
template <int PC>
__host__ __device__ __forceinline__ long long tc_abytes(int r1, int r3) {
  return (long long)TC_TILE * (r16(r1) + r16(r3)) * 2 * PC;
}

// Leaf gather of the prologue, a warp per entry row (lanes over the leaf's columns, no
// integer division per item), eight rows (24 loads) in flight per warp: the prologue's grid
// fits the GPU in one wave, so its time is one warp's chain of dependent loads, and more
// loads in flight shorten it.  Row e of c = sum_s w[e][m][s]
// U_m[row_s][:], zero for e >= nT.  TO_C1: into c1[e][node][0..63] (zero beyond r) in global
// scratch.  Otherwise into the A rows of the node (layout above): each lane splits its
// column's value into PC BF16 pieces, even lanes pair them with the next lane's into words
// and the first lane of each 8-column group gathers the group's four words into one 16-byte
// store, columns r .. r16 - 1 zero.  A prologue CTA holds ptile entries (32 or 128: a
// quarter of a tensor-core tile or a whole one; a_off: its first row in the tile's A rows);
// its four warps take eight rows per pass.
constexpr int PRO_THREADS = 128;
template <bool TO_C1, int PC>
__device__ __forceinline__ void gather_rows(void* dst, const float* __restrict__ U, int r, int m, int nT,
                                            const int* srow, const float* sw, int node, int a_off, int ptile) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rb16 = r16(r), ks = rb16 / 16;
  constexpr int RPI = 8;
  for (int e0 = RPI * warp; e0 < ptile; e0 += RPI * (PRO_THREADS / 32)) {
    int u[RPI][3];   // row offsets into U (a leaf has at most 128 rows of r <= 64 columns)
    float w[RPI][3];
#pragma unroll
    for (int k = 0; k < RPI; ++k) {
      const int e = e0 + k;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        u[k][q] = (e < nT ? srow[(e * 4 + m) * 3 + q] : 0) * r;
        w[k][q] = e < nT ? sw[(e * 4 + m) * 3 + q] : 0.f;
      }
    }
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 32) {
      if (!TO_C1 && c0 >= rb16) break;
      const int col = c0 + lane;
      float v[RPI][3];
#pragma unroll
      for (int k = 0; k < RPI; ++k)
#pragma unroll
        for (int q = 0; q < 3; ++q) v[k][q] = col < r ? __ldg(U + u[k][q] + col) : 0.f;
#pragma unroll
      for (int k = 0; k < RPI; ++k) {
        const float x = w[k][0] * v[k][0] + w[k][1] * v[k][1] + w[k][2] * v[k][2];
        if constexpr (TO_C1) {
          static_cast<float*>(dst)[(long long)(e0 + k) * 128 + node * 64 + col] = x;   // zero beyond r (v = 0)
        } else {
          float rest = x;
#pragma unroll
          for (int q = 0; q < PC; ++q) {
            const __nv_bfloat16 h = __float2bfloat16_rn(rest);
            rest -= __bfloat162float(h);
            const uint32_t lo = __bfloat16_as_ushort(h);
            const uint32_t word = lo | (__shfl_down_sync(0xffffffffu, lo, 1) << 16);
            const uint32_t w1 = __shfl_down_sync(0xffffffffu, word, 2), w2 = __shfl_down_sync(0xffffffffu, word, 4),
                           w3 = __shfl_down_sync(0xffffffffu, word, 6);
            if ((lane & 7) == 0 && col < rb16)
              static_cast<uint4*>(dst)[(q * ks * 2 + col / 8) * TC_TILE + a_off + e0 + k] = make_uint4(word, w1, w2, w3);
          }
        }
      }
    }
  }
}

// Prologue of the tensor-core evaluator, one CTA per ptile entries: 32 (a quarter of a
// tensor-core tile, so that a one-fibre launch of 16384 entries spreads over 512 CTAs) while
// the grid stays within two waves of four CTAs per SM, else 128: the feet, cells and
// weights, the four leaf gathers, the BF16 split of c2 of both nodes into the A rows of
// the tile and c1 of both nodes, all into global scratch.  A separate kernel so that these
// latency-bound steps run at several CTAs per SM and overlap one another, while the
// tensor-core kernel (one CTA per SM) starts its MMAs as soon as its warps have moved the A
// rows into tensor memory.
template <bool DEV, int PC>
__global__ void __launch_bounds__(PRO_THREADS, 4)   // 4 CTAs per SM: 592 >= the 512 CTAs of a 16384-entry fibre
k_tc_prologue(GridDesc g, HTView<float> ht_arg, const EvalParams<float>* __restrict__ P, EvalArgs a,
              TcScratch sc, int ptile) {
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
  // ptile entries from e0: rows a_off .. a_off + ptile - 1 of tensor-core tile `tile`
  const long long e0 = (long long)blockIdx.x * ptile;
  const long long tile = e0 / TC_TILE;
  const int a_off = (int)(e0 - tile * TC_TILE);
  const long long n_act = a.nact ? min(a.n, (long long)(*a.nact) * a.nper) : a.n;
  if (e0 >= n_act) return;
  const int nT = (int)min((long long)ptile, n_act - e0);
  const int tid = threadIdx.x;
  float* sw = reinterpret_cast<float*>(smem_raw);                     // ptile x 12
  int* srow = reinterpret_cast<int*>(sw + TC_TILE * 12);              // ptile x 12
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
    }
  }
  __syncthreads();
  // the tile's rows and weights to the scratch (for the correction epilogue), coalesced
  for (int i = tid; i < nT * 12; i += PRO_THREADS) {
    sc.rows[e0 * 12 + i] = srow[i];
    sc.w[e0 * 12 + i] = sw[i];
  }
  unsigned char* At = sc.a + tile * tc_abytes<PC>(ht.r[1], ht.r[3]);
  float* c1 = sc.c1 + e0 * 128;
  // c1 of both nodes and the A rows (split c2) of both nodes, straight to the scratch
  gather_rows<true, PC>(c1, ht.U[0], ht.r[0], 0, nT, srow, sw, 0, 0, ptile);
  gather_rows<true, PC>(c1, ht.U[2], ht.r[2], 2, nT, srow, sw, 1, 0, ptile);
  gather_rows<false, PC>(At, ht.U[1], ht.r[1], 1, nT, srow, sw, 0, a_off, ptile);
  gather_rows<false, PC>(At + (long long)TC_TILE * r16(ht.r[1]) * 2 * PC, ht.U[3], ht.r[3], 3, nT, srow, sw, 1,
                         a_off, ptile);
}

size_t tc_prologue_smem(const int*) { return (size_t)PRO_SMEM_BYTES; }

// entries per prologue CTA: 32 while the grid stays within two waves of four such CTAs per SM
// on 148 SMs, else 128
int tc_prologue_tile(long long n) { return (n + 31) / 32 <= 2 * 4 * 148 ? 32 : 128; }

template <bool DEV, int PC>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_sl_eval_tc(GridDesc g, HTView<float> ht_arg, CorrView corr_arg, const EvalParams<float>* __restrict__ P,
             EvalArgs a, const unsigned char* __restrict__ b12, const unsigned char* __restrict__ b34, int* err,
             TcScratch sc, const unsigned char* __restrict__ broot) {
  constexpr int SB = tc_sstages<PC>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // full, slot free (per shared slot); mma_done, drained (per tensor-memory slot); A operands
  // in tensor memory; root B; root MMAs; the two issuers' final commits
  __shared__ __align__(8) unsigned long long s_bar[2 * SB + 2 * TC_STAGES + 5];
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
  float* sout = reinterpret_cast<float*>(smem_raw + L.out);           // c_t[node][p][e]
  float* soutb = reinterpret_cast<float*>(smem_raw + L.outb);         // second partial sums (PC = 3)
  const uint32_t bslot = smem_u32(smem_raw + L.B);
  constexpr int NB0 = 2 * SB + 2 * TC_STAGES;
  const uint32_t full = smem_u32(&s_bar[0]), sfree = smem_u32(&s_bar[SB]), mdone = smem_u32(&s_bar[2 * SB]),
                 drained = smem_u32(&s_bar[2 * SB + TC_STAGES]), aready = smem_u32(&s_bar[NB0]),
                 rbar = smem_u32(&s_bar[NB0 + 1]), rdone = smem_u32(&s_bar[NB0 + 2]),
                 idone = smem_u32(&s_bar[NB0 + 3]);   // + 8 for the second issuer
  const long long abytes = tc_abytes<PC>(ht.r[1], ht.r[3]);

  const TcNode N0 = tc_node<PC>(ht.r[0], ht.r[1], ht.r12, (uint32_t)tc_acol<PC>(0), b12, 0);
  const TcNode N1 = tc_node<PC>(ht.r[2], ht.r[3], ht.r34, (uint32_t)tc_acol<PC>(1), b34, 64 * TC_TILE);
  const int nchunk = N0.nch + N1.nch;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < SB; ++i) {
      mbar_init(full + 8 * i, 1);
      mbar_init(sfree + 8 * i, 1);
    }
    for (int i = 0; i < TC_STAGES; ++i) {
      mbar_init(mdone + 8 * i, 1);
      mbar_init(drained + 8 * i, TC_CONSUMERS / 32);
    }
    mbar_init(aready, TC_CONSUMERS / 32);
    mbar_init(rbar, 1);
    mbar_init(rdone, 1);
    mbar_init(idone, 1);
    mbar_init(idone + 8, 1);
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
    const int s = j % SB;
    mbar_expect_tx(full + 8 * s, bytes);
    bulk_g2s(bslot + s * L.slot, N.bg + (long long)cl * N.w * N.rb16 * 2 * PC, bytes, full + 8 * s);
  };
  const bool copier = tid == TC_COPY_WARP * 32, issuer0 = tid == TC_MMA_WARP * 32,
             issuer = issuer0 || tid == TC_MMA2_WARP * 32;
  int n_copy = 0;
  if (copier)
    for (; n_copy < SB && n_copy < nchunk; ++n_copy) issue_copy(n_copy);

  // 2. c1 of node 0 into registers and the A operands of both nodes into tensor memory (from
  //    the prologue's scratch; the two warps of a lane quadrant take alternate 16-byte groups)
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
  if (warp < 8) {
    load_c1(0);
    const uint4* arow = reinterpret_cast<const uint4*>(sc.a + (long long)blockIdx.x * abytes);
    const int ng0 = PC * N0.ks * 2, ng1 = PC * N1.ks * 2;
    for (int gi = half; gi < ng0; gi += 2) tmem_st4(trow + N0.a_col + 4 * gi, arow[gi * TC_TILE + e_own]);
    for (int gi = half; gi < ng1; gi += 2)
      tmem_st4(trow + N1.a_col + 4 * gi, arow[(ng0 + gi) * TC_TILE + e_own]);
    tmem_wait_st();
    fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(aready);
  }

  // 3. the chunk stream
  if (issuer) {
    if (!wait_one(aready, 0)) {
      *(volatile int*)&s_abort = 1;
      atomicExch(err, 1);
    }
    for (int j = issuer0 ? 0 : 1; j < nchunk; j += 2) {
      if (*(volatile int*)&s_abort) break;
      const int s = j % SB, t = j % TC_STAGES;
      bool ok = wait_one(full + 8 * s, (uint32_t)(j / SB) & 1);
      if (ok && j >= TC_STAGES) ok = wait_one(drained + 8 * t, (uint32_t)((j - TC_STAGES) / TC_STAGES) & 1);
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
      const uint32_t dt = tmem + (uint32_t)(t * tc_w<PC>());
      const uint32_t a0 = tmem + N.a_col;
      const uint64_t b0 = tc_desc(bslot + s * L.slot);
      const uint32_t bk = (uint32_t)wc * 2;   // wc x 32 bytes / 16
      switch (N.ks) {
        case 1: issue_chunk<PC, 1>(dt, a0, b0, bk, idesc); break;
        case 2: issue_chunk<PC, 2>(dt, a0, b0, bk, idesc); break;
        case 3: issue_chunk<PC, 3>(dt, a0, b0, bk, idesc); break;
        default: issue_chunk<PC, 4>(dt, a0, b0, bk, idesc); break;
      }
      mma_commit(mdone + 8 * t);
      mma_commit(sfree + 8 * s);
    }
  } else if (copier) {
    for (int j = SB; j < nchunk; ++j) {
      if (*(volatile int*)&s_abort) break;
      const int s = j % SB;
      if (!wait_one(sfree + 8 * s, (uint32_t)((j - SB) / SB) & 1)) {
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
          float* so = sout + N.out_off + e_own;
          if constexpr (PC == 2) {
            switch (N.ra16) {
              case 16: drain_chunk<1>(creg, trow, sc, p0, p1, half, so); break;
              case 32: drain_chunk<2>(creg, trow, sc, p0, p1, half, so); break;
              case 48: drain_chunk<3>(creg, trow, sc, p0, p1, half, so); break;
              default: drain_chunk<4>(creg, trow, sc, p0, p1, half, so); break;
            }
          } else {
            float* sob = soutb + N.out_off + e_own;
            switch (N.ra16) {
              case 16: drain_chunk3<1>(creg, trow, sc, p0, p1, half, so, sob); break;
              case 32: drain_chunk3<2>(creg, trow, sc, p0, p1, half, so, sob); break;
              case 48: drain_chunk3<3>(creg, trow, sc, p0, p1, half, so, sob); break;
              default: drain_chunk3<4>(creg, trow, sc, p0, p1, half, so, sob); break;
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
  if (copier)
    for (int k = n_copy - SB < 0 ? 0 : n_copy - SB; k < n_copy; ++k) wait_one(full + 8 * (k % SB), (uint32_t)(k / SB) & 1);
  // each issuer's MMAs (one single-phase barrier per issuer, committed after all of them:
  // a slot barrier of the stream could have moved on by two phases, the other issuer's)
  if (issuer) {
    const uint32_t ib = idone + (issuer0 ? 0u : 8u);
    mma_commit(ib);
    wait_one(ib, 0);
  }
  __syncwarp();
  fence_before();
  __syncthreads();
  fence_after();
  const bool ok = *(volatile int*)&s_abort == 0;

  if (ok) {
    // 4. root on the tensor cores: T[e][p] = sum_q c34[e][q] Broot[p][q], a [128 x r34] x
    //    [r34 x r12] GEMM (c34 split into PC BF16 pieces as the A operand in node 0's A
    //    columns of tensor memory, the pre-split Broot bulk-copied into the freed B ring),
    //    then sum_p c12[e][p] T[e][p] per entry; the two warps of a lane quadrant take p < 32
    //    and p >= 32
    const int rl = ht.r12, rr = ht.r34;
    const int n16 = r16(rl), kr16 = r16(rr), ksr = kr16 / 16;
    const uint32_t rb_addr = bslot;
    const uint32_t rbytes = (uint32_t)(n16 * kr16 * 2 * PC);
    bool root_mma = false;
    if (copier) {
      mbar_expect_tx(rbar, rbytes);
      bulk_g2s(rb_addr, broot, rbytes, rbar);
    }
    float c12h[32];
    if (warp < 8) {
      float c34[64];
      const float* s34 = sout + 64 * TC_TILE + e_own;
      const float* s12 = sout + (half * 32) * TC_TILE + e_own;
#pragma unroll
      for (int q = 0; q < 64; ++q) c34[q] = q < rr ? s34[q * TC_TILE] : 0.f;
#pragma unroll
      for (int i = 0; i < 32; ++i) c12h[i] = s12[i * TC_TILE];
      if constexpr (PC == 3) {
        // the second partial sums of nodes whose a-range spans both halves of a chunk
        if (N1.ra16 > 32) {
          const float* b34p = soutb + 64 * TC_TILE + e_own;
#pragma unroll
          for (int q = 0; q < 64; ++q)
            if (q < rr) c34[q] += b34p[q * TC_TILE];
        }
        if (N0.ra16 > 32) {
          const float* b12p = soutb + (half * 32) * TC_TILE + e_own;
#pragma unroll
          for (int i = 0; i < 32; ++i)
            if (half * 32 + i < rl) c12h[i] += b12p[i * TC_TILE];
        }
      }
      // row e_own of the A operand into node 0's A columns: this warp's K groups of 8
#pragma unroll
      for (int kg = 0; kg < 8; ++kg) {
        if ((kg & 1) == half && kg * 8 < kr16) {
          float x[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) x[j] = c34[kg * 8 + j];
          uint4 pcs[PC];
          split8<PC>(x, pcs);
#pragma unroll
          for (int q = 0; q < PC; ++q) tmem_st4(trow + N0.a_col + 4 * (q * ksr * 2 + kg), pcs[q]);
        }
      }
      tmem_wait_st();
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (issuer0) {
      if (wait_one(rbar, 0)) {
        root_mma = true;
        fence_after();
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n16 >> 3) << 17) |
                               ((uint32_t)(TC_TILE >> 4) << 24);
        const uint32_t a0 = tmem + N0.a_col;
        const uint64_t b0 = tc_desc(rb_addr);
        const uint32_t bk = (uint32_t)n16 * 2;
        switch (ksr) {
          case 1: issue_chunk<PC, 1>(tmem, a0, b0, bk, idesc); break;
          case 2: issue_chunk<PC, 2>(tmem, a0, b0, bk, idesc); break;
          case 3: issue_chunk<PC, 3>(tmem, a0, b0, bk, idesc); break;
          default: issue_chunk<PC, 4>(tmem, a0, b0, bk, idesc); break;
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
    if (issuer0 && root_mma) wait_one(rdone, 0);
    __syncthreads();
    // 5. correction and residual epilogue
    if (tid < nT) {
      double val = sval[tid];
      if (corr.has) val += (double)correction_rw_ft<2>(g, corr, sc.rows + (e0 + tid) * 12, sc.w + (e0 + tid) * 12);
      const long long e = e0 + tid;
      if (a.X) {
        const unsigned eu = (unsigned)e, nper = (unsigned)a.nper;   // below 2^31: 32-bit division
        const unsigned fib = nper ? eu / nper : 0u;
        const long long piv = (long long)a.pivot[fib];
        const long long ey = (long long)(nper ? eu - fib * nper : eu);
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
  const int mp = PRO_SMEM_BYTES;
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
    const int pt = tc_prologue_tile(a.n);
    const long long blocks = (a.n + TC_TILE - 1) / TC_TILE, pblocks = (a.n + pt - 1) / pt;
    if (pieces == 3) {
      slar::count_launch(), k_tc_prologue<false, 3><<<(unsigned)pblocks, PRO_THREADS, smp, s>>>(g, ht, nullptr, a, sc,
                                                                                             pt);
      slar::count_launch(), k_sl_eval_tc<false, 3><<<(unsigned)blocks, TC_THREADS, sm, s>>>(g, ht, corr, nullptr, a,
                                                                                           p12, p34, err, sc, broot);
    } else {
      slar::count_launch(), k_tc_prologue<false, 2><<<(unsigned)pblocks, PRO_THREADS, smp, s>>>(g, ht, nullptr, a, sc,
                                                                                             pt);
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
  const int pt = tc_prologue_tile(a.n);
  const long long blocks = (a.n + TC_TILE - 1) / TC_TILE, pblocks = (a.n + pt - 1) / pt;
  const unsigned char* p12 = static_cast<const unsigned char*>(b12);
  const unsigned char* p34 = static_cast<const unsigned char*>(b34);
  const size_t smp = (size_t)PRO_SMEM_BYTES;
  if (pieces == 3) {
    slar::count_launch(), k_tc_prologue<true, 3><<<(unsigned)pblocks, PRO_THREADS, smp, s>>>(g, HTView<float>{}, P, a,
                                                                                         sc, pt);
    slar::count_launch(), k_sl_eval_tc<true, 3><<<(unsigned)blocks, TC_THREADS, sm, s>>>(
        g, HTView<float>{}, CorrView{}, P, a, p12, p34, err, sc, broot);
  } else {
    slar::count_launch(), k_tc_prologue<true, 2><<<(unsigned)pblocks, PRO_THREADS, smp, s>>>(g, HTView<float>{}, P, a,
                                                                                         sc, pt);
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
