// Tensor-core complex GEMM for sm_103a (tcgen05, accumulator in tensor
// memory) with FP32 accuracy from TF32 products: every FP32 operand value x is
// split into x_hi = tf32(x) and x_lo = tf32(x - x_hi), both rounded to
// nearest, so x = x_hi + x_lo to about 2^-22 |x|; each real product is the sum
// of the four TF32 products A_hi B_hi + A_hi B_lo + A_lo B_hi + A_lo B_lo
// (each exact in the FP32 accumulator's precision).
//
// One CTA of 128 threads (one warpgroup) computes a 128 x 128 real tile.  Per
// 32-wide real K chunk the threads stage A and B^T, split into hi and lo, in
// shared memory in the canonical K-major 128-byte-swizzled layout (8-row
// atoms of 1024 bytes; the 16-byte chunk c of row r sits at chunk c ^ (r mod
// 8)); one thread issues the 4 x 4 tcgen05.mma (M 128, N 128, K 8) and
// commits them to an mbarrier that every thread waits on with a bounded spin.
// After each chunk the threads read its product with tcgen05.ld (warp w owns
// rows 32w..32w+31) and add it to FP32 sums in registers.  A wait that runs out sets *err; the accumulator is released
// in every case.
#pragma once

#include <stdint.h>

namespace mpsv {
namespace tc {

constexpr int kBM = 128, kBN = 128, kBK = 32;
constexpr int kThreads = 128;
constexpr uint32_t kTmemCols = 128;
constexpr int kTileBytes = kBM * kBK * 4;  // 16 KB per operand tile (hi or lo)
constexpr long long kSpinLimit = 1ll << 26;
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s: a tile's MMAs take microseconds

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// K-major SWIZZLE_128B shared-memory matrix descriptor (tcgen05): start
// address >> 4 in bits 0-13, leading-byte offset (unused for this layout) in
// 16-29, stride-byte offset (1024 B between 8-row atoms) >> 4 in 32-45, the
// descriptor version 1 in bits 46-47, swizzle mode 2 (128 B) in bits 61-63.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9 and 10-12 = 2), both K-major, N >> 3 in bits 17-22, M >> 4 in 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (row, k) of a K-major 128B-swizzled tile, 0 <= k < 32
__device__ __forceinline__ uint32_t swz_offset(int row, int k) {
  const int chunk = (k >> 2) ^ (row & 7);
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + chunk * 16 + (k & 3) * 4);
}

__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm volatile("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for the phase with parity `parity` to complete; false once
// kWaitNs nanoseconds (or kSpinLimit polls) have passed without it.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const uint64_t t0 = global_ns();
  for (long long i = 0; i < kSpinLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((i & 255) == 255 && global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

// 32 lanes x 16 consecutive 32-bit columns of tensor memory into v (this warp's lane quarter)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// Complex GEMM on the tensor cores.  For problem z the product is
// C[m][n] = sum_k a(z, m, k) b(z, k, n) (complex FP32, M x N x K from
// prob.dims), computed as the real GEMM C_r = A_r B_r with A_r[m][2k + t] =
// (Re, Im)_t of a and B_r the 2 x 2 real embedding [[Re b, Im b], [-Im b,
// Re b]] of each b, so C_r[m][2n + u] = (Re, Im)_u of C.  A CTA computes 128
// rows x 64 complex columns; blockIdx.x = z * tiles_n + n-tile, blockIdx.y =
// m-tile.  The loaders of Prob give a() and b() for any stored layout
// (transposes, conjugation and phases included), so no operand is copied
// into an intermediate layout in global memory.
template <class Prob>
__global__ void __launch_bounds__(kThreads, 1) cgemm_kernel(Prob prob, int tiles_n, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* tA_hi = base;
  unsigned char* tA_lo = base + kTileBytes;
  unsigned char* tB_hi = base + 2 * kTileBytes;
  unsigned char* tB_lo = base + 3 * kTileBytes;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base_s;
  __shared__ int s_fail;

  const int z = blockIdx.x / tiles_n;
  const int nt = blockIdx.x % tiles_n;
  int M, N, K;
  prob.dims(z, M, N, K);
  const int m0 = blockIdx.y * kBM, n0 = nt * (kBN / 2);
  if (m0 >= M || n0 >= N || K <= 0) return;  // the whole CTA, before any tensor-memory use

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base_s;
  const uint32_t idesc = idesc_tf32(kBM, kBN);
  constexpr int kKC = kBK / 2;  // complex K per chunk

  uint32_t phase = 0;
  bool ok = true;
  float acc[kBN];
#pragma unroll
  for (int j = 0; j < kBN; ++j) acc[j] = 0.f;
  const int nk = (K + kKC - 1) / kKC;
  for (int kc = 0; kc < nk && ok; ++kc) {
    const int k0 = kc * kKC;
    // A: 128 rows x 16 complex -> real columns (2k, 2k + 1) = (Re, Im)
    for (int e = tid; e < kBM * kKC; e += kThreads) {
      const int r = e / kKC, kk = e % kKC;
      const int gm = m0 + r, gk = k0 + kk;
      float2 v = make_float2(0.f, 0.f);
      if (gm < M && gk < K) v = prob.a(z, gm, gk);
      const float rh = tf32_hi(v.x), ih = tf32_hi(v.y);
      const uint32_t o0 = swz_offset(r, 2 * kk), o1 = swz_offset(r, 2 * kk + 1);
      *reinterpret_cast<float*>(tA_hi + o0) = rh;
      *reinterpret_cast<float*>(tA_lo + o0) = tf32_hi(v.x - rh);
      *reinterpret_cast<float*>(tA_hi + o1) = ih;
      *reinterpret_cast<float*>(tA_lo + o1) = tf32_hi(v.y - ih);
    }
    // B^T: 64 complex columns n x 16 complex k -> 2 x 2 real blocks
    for (int e = tid; e < (kBN / 2) * kKC; e += kThreads) {
      const int nn = e / kKC, kk = e % kKC;
      const int gn = n0 + nn, gk = k0 + kk;
      float2 v = make_float2(0.f, 0.f);
      if (gn < N && gk < K) v = prob.b(z, gk, gn);
      const float rh = tf32_hi(v.x), ih = tf32_hi(v.y), nih = -ih;
      const float rl = tf32_hi(v.x - rh), il = tf32_hi(v.y - ih);
      const uint32_t o00 = swz_offset(2 * nn, 2 * kk), o01 = swz_offset(2 * nn, 2 * kk + 1);
      const uint32_t o10 = swz_offset(2 * nn + 1, 2 * kk), o11 = swz_offset(2 * nn + 1, 2 * kk + 1);
      *reinterpret_cast<float*>(tB_hi + o00) = rh;
      *reinterpret_cast<float*>(tB_lo + o00) = rl;
      *reinterpret_cast<float*>(tB_hi + o01) = nih;
      *reinterpret_cast<float*>(tB_lo + o01) = -il;
      *reinterpret_cast<float*>(tB_hi + o10) = ih;
      *reinterpret_cast<float*>(tB_lo + o10) = il;
      *reinterpret_cast<float*>(tB_hi + o11) = rh;
      *reinterpret_cast<float*>(tB_lo + o11) = rl;
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint64_t dAh = smem_desc(smem_u32(tA_hi)), dAl = smem_desc(smem_u32(tA_lo));
      const uint64_t dBh = smem_desc(smem_u32(tB_hi)), dBl = smem_desc(smem_u32(tB_lo));
#pragma unroll
      for (int ks = 0; ks < kBK / 8; ++ks) {
        const uint64_t adv = (uint64_t)((ks * 32) >> 4);  // 8 tf32 = 32 bytes along K
        mma_tf32(tmem, dAh + adv, dBh + adv, idesc, ks > 0 ? 1u : 0u);
        mma_tf32(tmem, dAh + adv, dBl + adv, idesc, 1u);
        mma_tf32(tmem, dAl + adv, dBh + adv, idesc, 1u);
        mma_tf32(tmem, dAl + adv, dBl + adv, idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&mbar)));
    }
    if (!mbar_wait(&mbar, phase)) s_fail = 1;
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    if (s_fail) {
      ok = false;
    } else {
      // the chunk's partial product joins the FP32 sum in registers (rounded
      // to nearest), which keeps the tensor cores' own accumulation chains
      // to one chunk of 32 real K
#pragma unroll
      for (int c0 = 0; c0 < kBN; c0 += 16) {
        uint32_t v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[c0 + j] += __uint_as_float(v[j]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;");  // loads done before the next chunk's MMAs
    }
  }

  if (ok) {
    const int row = m0 + warp * 32 + lane;  // warp w holds accumulator rows 32w .. 32w+31
    if (row < M) {
#pragma unroll
      for (int j = 0; j < kBN / 2; ++j) {
        const int col = n0 + j;
        if (col < N) prob.store(z, row, col, make_float2(acc[2 * j], acc[2 * j + 1]));
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

constexpr size_t kSmemBytes = 4 * kTileBytes + 1024;

}  // namespace tc
}  // namespace mpsv
