// TMA-fed tensor-core complex GEMM for sm_103a (tcgen05, accumulators in
// tensor memory) with split products: the theta contraction (Methods, "MPS
// algorithm for quantum circuit simulation": C = Q (B_q B_{q+1}), Eq. tildeC)
// and the new left site tensor (Eq. Bl: B~_q = C V^dagger) of complex64
// states at large bond dimensions.
//
// Complex arithmetic.  A complex GEMM D = A B (M x N x K) runs as one real
// GEMM D_r = A_r B_e^T of M x 2N x 2K: A_r is A's interleaved (re, im) data
// read as reals (row m, real column 2k + t), and B_e is the 2 x 2 real
// embedding of B, row 2n = (Re b, -Im b) and row 2n + 1 = (Im b, Re b) along
// 2k + t, so that D_r[m][2n + u] is component u of D[m][n] - four real
// multiply-adds per complex one, as in the 4M form, with D written back in
// the library's interleaved layout.
//
// Split products.  Each real operand value x is held as x_hi + x_lo with
// x_hi = rna_tf32(x) and x_lo = rna_tf32(x - x_hi) (TF32 mode) or as
// x_hi = rn_bf16(x), x_lo = rn_bf16(x - x_hi) (BF16 mode); every real
// product is A_hi B_hi + A_hi B_lo + A_lo B_hi (three tensor-core products,
// the lo x lo term is below the target accuracy).  TF32 pieces keep
// 22 bits of x (about FP32 accuracy); BF16 pieces keep 16 bits at twice the
// tensor-core rate.  A split kernel writes the pieces once per operand into
// zero-padded K-major planes, which the GEMM loads with TMA.
//
// GEMM kernel.  One CTA computes a 128-row x 64-complex-column tile with six
// warps: warp 0 issues the TMA loads of a three-stage shared-memory ring
// (per stage: 128 rows x 128 bytes of A_hi, A_lo, B_hi and B_lo, 128-byte
// swizzled, 64 KB), warp 1 allocates tensor memory and issues the
// tcgen05.mma of each 128-byte K chunk (12 TF32 or 12 BF16 instructions, 3
// products each) into one of two 128-column accumulators, and warps 2-5 drain
// each finished accumulator (kDrain chunks: the tensor cores' own
// accumulation chain stays that long) with tcgen05.ld into FP32 registers
// and, at the end, apply the epilogue of the contraction, staging the rows
// in shared memory so that the global stores coalesce.  mbarriers order every hand-over;
// every wait is bounded (2 s): a wait that runs out raises a CTA-wide abort
// flag, every role stops issuing, the error flag is set and tensor memory is
// released.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"

namespace mpsv {
namespace tma {

constexpr int kBM = 128;         // rows per CTA (one accumulator lane per row)
constexpr int kBNr = 128;        // real columns per CTA (64 complex)
constexpr int kBNc = kBNr / 2;   // complex columns per CTA
constexpr int kChunkBytes = 128; // bytes of K per stage (one swizzle row)
constexpr int kStages = 3;
constexpr int kPlaneBytes = kBM * kChunkBytes;  // 16 KB: one operand piece of one stage
constexpr int kStageBytes = 4 * kPlaneBytes;    // A_hi, A_lo, B_hi, B_lo
constexpr int kThreads = 192;
constexpr uint32_t kTmemCols = 2 * kBNr;        // two chunk accumulators
constexpr size_t kSmemBytes = (size_t)kStages * kStageBytes + 1024;
constexpr uint64_t kWaitNs = 2000000000ull;
// K chunks accumulated in one tensor-memory buffer before the epilogue warps
// drain it into FP32 registers (the length of the tensor cores' own
// accumulation chain, in chunks)
constexpr int kDrain = 4;

enum Mode { kTF32 = 0, kBF16 = 1 };

// Element size and K per MMA of a mode; padded real K is a multiple of the
// chunk's element count (32 TF32 or 64 BF16 values).
template <int M> struct ModeTraits;
template <> struct ModeTraits<kTF32> {
  using T = float;
  static constexpr int kElemsPerChunk = 32;
  static constexpr int kMmaK = 8;  // elements per tcgen05.mma (32 bytes)
};
template <> struct ModeTraits<kBF16> {
  using T = uint16_t;
  static constexpr int kElemsPerChunk = 64;
  static constexpr int kMmaK = 16;
};

__host__ __device__ inline int pad_k(int kr, int mode) {
  const int e = mode == kTF32 ? 32 : 64;
  return (kr + e - 1) / e * e;
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t su32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count));
}

__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}

// Bounded wait for the phase of parity `par`; false when *abort is raised or
// kWaitNs passed (then *abort is raised here).
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t par, volatile int* abort) {
  // (a wait whose *abort is a local zero is only bounded by time)
  const uint32_t a = su32(b);
  const uint64_t t0 = now_ns();
  for (uint32_t i = 0;; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(par)
        : "memory");
    if (done) return true;
    if ((i & 63) == 63) {
      if (*abort) return false;
      if (now_ns() - t0 > kWaitNs) {
        *abort = 1;
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(su32(bar))
      : "memory");
}

// K-major SWIZZLE_128B shared-memory descriptor: start >> 4 (bits 0-13),
// leading-byte offset 1 (unused by this layout, bits 16-29), stride-byte
// offset 1024 >> 4 between 8-row atoms (bits 32-45), version 1 (bits 46-47),
// swizzle mode 2 = 128 B (bits 61-63).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptors (D FP32 in bits 4-5; A, B formats in 7-9 and
// 10-12; both K-major; N >> 3 in 17-22; M >> 4 in 24-28).  kind::tf32:
// format 2 = TF32.  kind::f16: format 1 = BF16.
__host__ __device__ constexpr uint32_t idesc_for(int mode, int M, int N) {
  return (1u << 4) | ((mode == kTF32 ? 2u : 1u) << 7) | ((mode == kTF32 ? 2u : 1u) << 10) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int M>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (M == kTF32)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}

// 32 lanes x 32 consecutive FP32 columns of tensor memory.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float rna_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// hi / lo pieces of one real value in the mode's element type
template <int M> struct Split;
template <> struct Split<kTF32> {
  static __device__ __forceinline__ void run(float x, float& hi, float& lo) {
    hi = rna_tf32(x);
    lo = rna_tf32(x - hi);
  }
};
template <> struct Split<kBF16> {
  static __device__ __forceinline__ void run(float x, uint16_t& hi, uint16_t& lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
  }
};

// ---------------------------------------------------------------------------
// split kernel (operand planes: rows x ld elements, K-major, zero-padded)
// ---------------------------------------------------------------------------

// Four consecutive real values of one plane row (16 bytes of TF32, 8 of BF16).
template <int M> struct Quad;
template <> struct Quad<kTF32> {
  static __device__ __forceinline__ void store(float* p, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
  }
};
template <> struct Quad<kBF16> {
  static __device__ __forceinline__ void store(uint16_t* p, uint16_t a, uint16_t b, uint16_t c, uint16_t d) {
    *reinterpret_cast<uint2*>(p) = make_uint2((uint32_t)a | ((uint32_t)b << 16), (uint32_t)c | ((uint32_t)d << 16));
  }
};

// Both operands of one GEMM in one launch.  Blocks [0, a_blocks) write the
// A planes, the others the B planes.
//  * A (SrcA: dims(rows, K), a(r, k)): row r, real columns 2k + t; a thread
//    handles two consecutive complex K values (four real columns: 16- or
//    8-byte stores along a row), so reads and writes run along K.
//  * B (SrcB: dims(N_pad, K), b(k, n, ok)): the 2 x 2 real embedding, row 2n =
//    (Re b, -Im b) and row 2n + 1 = (Im b, Re b) along 2k + t; padding
//    columns (ok cleared) give zero rows.  Where consecutive n of one k are
//    consecutive in memory (SrcB::kAlongN, the theta's right site tensor) a
//    block stages a 32 k x 32 n tile in shared memory, read along n and
//    written along K; otherwise threads run along K as for A.
// Real columns from 2K up to the chunk boundary are written as zeros; sizes
// come from device memory, so the grid is sized for the capacities.
template <int M>
__device__ __forceinline__ void store_b_pair(typename ModeTraits<M>::T* bhi, typename ModeTraits<M>::T* blo, int ld,
                                             int n, int k, float2 v0, float2 v1) {
  using T = typename ModeTraits<M>::T;
  T hr0, lr0, hi0, li0, hn0, ln0, hr1, lr1, hi1, li1, hn1, ln1;
  Split<M>::run(v0.x, hr0, lr0);
  Split<M>::run(v0.y, hi0, li0);
  Split<M>::run(-v0.y, hn0, ln0);
  Split<M>::run(v1.x, hr1, lr1);
  Split<M>::run(v1.y, hi1, li1);
  Split<M>::run(-v1.y, hn1, ln1);
  const size_t o0 = (size_t)(2 * n) * ld + 2 * k, o1 = o0 + ld;
  Quad<M>::store(bhi + o0, hr0, hn0, hr1, hn1);
  Quad<M>::store(bhi + o1, hi0, hr0, hi1, hr1);
  Quad<M>::store(blo + o0, lr0, ln0, lr1, ln1);
  Quad<M>::store(blo + o1, li0, lr0, li1, lr1);
}

constexpr int kSplitTile = 32;  // k and n extent of a staged B tile

template <int M, class SrcA, class SrcB>
__global__ void __launch_bounds__(256) split_ab_kernel(SrcA sa, SrcB sb, int ld, int a_blocks,
                                                        typename ModeTraits<M>::T* __restrict__ ahi,
                                                        typename ModeTraits<M>::T* __restrict__ alo,
                                                        typename ModeTraits<M>::T* __restrict__ bhi,
                                                        typename ModeTraits<M>::T* __restrict__ blo) {
  using T = typename ModeTraits<M>::T;
  __shared__ float2 tile[kSplitTile][kSplitTile + 1];
  if ((int)blockIdx.x < a_blocks) {
    int rows, Ka;
    sa.dims(rows, Ka);
    const int pa = pad_k(2 * Ka, M) / 4;  // k pairs per row
    const long long na = (long long)rows * pa;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < na; e += (long long)a_blocks * blockDim.x) {
      const int r = (int)(e / pa), k = 2 * (int)(e % pa);
      const float2 v0 = k < Ka ? sa(r, k) : make_float2(0.f, 0.f);
      const float2 v1 = k + 1 < Ka ? sa(r, k + 1) : make_float2(0.f, 0.f);
      T h[4], l[4];
      Split<M>::run(v0.x, h[0], l[0]);
      Split<M>::run(v0.y, h[1], l[1]);
      Split<M>::run(v1.x, h[2], l[2]);
      Split<M>::run(v1.y, h[3], l[3]);
      const size_t o = (size_t)r * ld + 2 * k;
      Quad<M>::store(ahi + o, h[0], h[1], h[2], h[3]);
      Quad<M>::store(alo + o, l[0], l[1], l[2], l[3]);
    }
    return;
  }
  int npad, Kb;
  sb.dims(npad, Kb);
  const int pb = pad_k(2 * Kb, M) / 4;  // k pairs per embedded row
  const int bblk = (int)blockIdx.x - a_blocks, nbblk = (int)gridDim.x - a_blocks;
  if constexpr (SrcB::kAlongN) {
    const int kpad = 2 * pb, tn = (npad + kSplitTile - 1) / kSplitTile, tk = (kpad + kSplitTile - 1) / kSplitTile;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = bblk; t < tn * tk; t += nbblk) {
      const int n0 = (t % tn) * kSplitTile, k0 = (t / tn) * kSplitTile;
#pragma unroll
      for (int i = 0; i < kSplitTile / 8; ++i) {
        const int kl = w + 8 * i, k = k0 + kl, n = n0 + lane;
        bool ok = false;
        float2 v = make_float2(0.f, 0.f);
        if (k < Kb && n < npad) v = sb(k, n, ok);
        tile[kl][lane] = ok ? v : make_float2(0.f, 0.f);
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < (kSplitTile * kSplitTile / 2) / 256; ++i) {
        const int item = (int)threadIdx.x + 256 * i;
        const int nl = item / (kSplitTile / 2), kp = item % (kSplitTile / 2);
        const int n = n0 + nl, k = k0 + 2 * kp;
        if (n < npad && k < kpad) store_b_pair<M>(bhi, blo, ld, n, k, tile[2 * kp][nl], tile[2 * kp + 1][nl]);
      }
      __syncthreads();
    }
  } else {
    const long long nb = (long long)npad * pb;
    for (long long e = bblk * (long long)blockDim.x + threadIdx.x; e < nb; e += (long long)nbblk * blockDim.x) {
      const int n = (int)(e / pb), k = 2 * (int)(e % pb);
      bool ok0 = false, ok1 = false;
      float2 v0 = make_float2(0.f, 0.f), v1 = v0;
      if (k < Kb) v0 = sb(k, n, ok0);
      if (k + 1 < Kb) v1 = sb(k + 1, n, ok1);
      if (!ok0) v0 = make_float2(0.f, 0.f);
      if (!ok1) v1 = make_float2(0.f, 0.f);
      store_b_pair<M>(bhi, blo, ld, n, k, v0, v1);
    }
  }
}

// ---------------------------------------------------------------------------
// the GEMM
// ---------------------------------------------------------------------------
// Operand maps: A planes [rows_cap][ld], B planes [2 N_cap][ld] (each a 2-D
// tensor map with a 128-byte x 128-row box).  CTA (bx, by) computes rows
// 128 by .. and logical complex columns 64 bx ..; the grid is sized for the
// capacities and the epilogue functor's dims() gives the actual rows, real K
// and logical columns (read from device memory).
//
// Epilogue functor interface (both calls made by every lane of a warp, rows
// past the actual count included):
//  * values(row, nbase, acc, v): from acc[2c + u] = component u of complex
//    column nbase + c (c < 64) of this lane's row, the 64 complex outputs of
//    the row, v[32 h + e] = entry e of output run h; rows r and r ^ 1 sit in
//    lanes l and l ^ 1 of one warp, for exchanges between neighbouring rows;
//  * run(row, nbase, h, count): where output run h of the row starts in
//    global memory (32 consecutive complex values, of which the first count
//    exist), or nullptr for a row past the actual count.
// The epilogue warps stage their rows' outputs in the (then idle) pipeline
// shared memory and write each run with consecutive lanes, so the stores
// coalesce.
template <int M, class Epi>
__global__ void __launch_bounds__(kThreads, 1)
    cgemm_tma_kernel(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
                     const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo, Epi epi,
                     int* __restrict__ err) {
  using TR = ModeTraits<M>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], tfull[2], tempty[2], drained;
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kBM;
  int rows, kr, ncols;  // actual rows, real K (2 x complex K), logical complex columns (padded to 64)
  epi.dims(rows, kr, ncols);
  const int nkc = (kr + TR::kElemsPerChunk - 1) / TR::kElemsPerChunk;
  // whole CTAs past the actual sizes leave before any barrier or tensor memory use
  if (m0 >= rows || (int)blockIdx.x * kBNc >= ncols || nkc == 0) return;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      bar_init(&full[s], 1);
      bar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      bar_init(&tfull[b], 1);
      bar_init(&tempty[b], 4);  // one arrival per epilogue warp
    }
    bar_init(&drained, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base_s)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_s;
  const int n0r = blockIdx.x * kBNr;  // first real B row (embedded column) of the tile

  if (warp == 0) {
    // ---- TMA producer
    if (lane == 0) {
      int issued = 0;
      for (int kc = 0; kc < nkc; ++kc) {
        const int s = kc % kStages;
        const uint32_t par = ((kc / kStages) & 1) ^ 1;
        if (!bar_wait(&empty[s], par, &abort_s)) break;
        unsigned char* st = base + (size_t)s * kStageBytes;
        bar_expect_tx(&full[s], kStageBytes);
        const int x = kc * TR::kElemsPerChunk;  // element coordinate along K (x 4 or 2 bytes: 128-byte aligned)
        tma_load_2d(st, &mAhi, x, m0, &full[s]);
        tma_load_2d(st + kPlaneBytes, &mAlo, x, m0, &full[s]);
        tma_load_2d(st + 2 * kPlaneBytes, &mBhi, x, n0r, &full[s]);
        tma_load_2d(st + 3 * kPlaneBytes, &mBlo, x, n0r, &full[s]);
        issued = kc + 1;
      }
      // no copy may still be landing in shared memory when the CTA leaves:
      // wait (bounded by time alone) for the last stages issued; on the
      // normal path the MMA warp has consumed them already
      for (int kc = max(0, issued - kStages); kc < issued; ++kc) {
        int never = 0;
        bar_wait(&full[kc % kStages], (kc / kStages) & 1, &never);
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_for(M, kBM, kBNr);
      constexpr int kSub = kChunkBytes / (TR::kMmaK * (int)sizeof(typename TR::T));  // MMAs per chunk per product
      for (int kc = 0; kc < nkc; ++kc) {
        const int s = kc % kStages;
        const int grp = kc / kDrain, b = grp & 1;
        const bool first = kc % kDrain == 0, last = kc % kDrain == kDrain - 1 || kc == nkc - 1;
        if (!bar_wait(&full[s], (kc / kStages) & 1, &abort_s)) break;
        if (first && !bar_wait(&tempty[b], ((grp >> 1) & 1) ^ 1, &abort_s)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = su32(base + (size_t)s * kStageBytes);
        const uint64_t dAh = sdesc(st), dAl = sdesc(st + kPlaneBytes);
        const uint64_t dBh = sdesc(st + 2 * kPlaneBytes), dBl = sdesc(st + 3 * kPlaneBytes);
        const uint32_t d = tmem + (uint32_t)(b * kBNr);
#pragma unroll
        for (int ks = 0; ks < kSub; ++ks) {
          const uint64_t adv = (uint64_t)((ks * TR::kMmaK * (int)sizeof(typename TR::T)) >> 4);
          mma<M>(d, dAh + adv, dBh + adv, idesc, (first && ks == 0) ? 0u : 1u);
          mma<M>(d, dAh + adv, dBl + adv, idesc, 1u);
          mma<M>(d, dAl + adv, dBh + adv, idesc, 1u);
        }
        mma_commit(&empty[s]);        // the stage's operands are free once these MMAs are done
        if (last) mma_commit(&tfull[b]);  // and the group's accumulator is ready
      }
      // every MMA issued before this point has completed once `drained`
      // fires; this wait ignores the abort flag (tensor memory is released
      // after it), bounded all the same
      mma_commit(&drained);
      int never = 0;
      bar_wait(&drained, 0, &never);
    }
  } else {
    // ---- epilogue warps: drain group accumulators into FP32 registers
    const int quarter = warp & 3;  // tensor-memory lane quarter this warp may access
    const int row = m0 + quarter * 32 + lane;
    float acc[kBNr];
#pragma unroll
    for (int j = 0; j < kBNr; ++j) acc[j] = 0.f;
    bool ok = true;
    const int ngrp = (nkc + kDrain - 1) / kDrain;
    for (int grp = 0; grp < ngrp && ok; ++grp) {
      const int b = grp & 1;
      // warp-uniform: tcgen05.ld below needs every lane
      if (!__all_sync(0xffffffffu, bar_wait(&tfull[b], (grp >> 1) & 1, &abort_s))) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * kBNr);
#pragma unroll
      for (int c0 = 0; c0 < kBNr; c0 += 32) {
        float v[32];
        tmem_ld32(ta + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[c0 + j] += v[j];
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) bar_arrive(&tempty[b]);
    }
    ok = ok && !abort_s;
    if (ok) {
      // Every MMA has completed (the last group's commit), so the pipeline
      // stages hold no operand still being read and every TMA copy has
      // landed: each epilogue warp stages its 32 rows x 64 outputs there.
      const int nbase = blockIdx.x * kBNc;
      float2 v[64];
      epi.values(row, nbase, acc, v);
      constexpr int kPad = 65;  // row stride in complex values (conflict-light staging writes)
      float2* stage = reinterpret_cast<float2*>(base) + (size_t)(warp - 2) * 32 * kPad;
#pragma unroll
      for (int e = 0; e < 64; ++e) stage[lane * kPad + e] = v[e];
      __syncwarp();
      for (int r = 0; r < 32; ++r) {
        const int rr = m0 + quarter * 32 + r;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          int count = 0;
          float2* dst = epi.run(rr, nbase, h, count);
          if (dst != nullptr && lane < count) dst[lane] = stage[r * kPad + 32 * h + lane];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (abort_s && threadIdx.x == 0) atomicExch(err, 1);
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

}  // namespace tma
}  // namespace mpsv
