// Tensor-core theta and new-left-tensor contractions of a two-qubit gate for
// complex64 states in the split-product precision modes (MPS_PREC_TF32X3,
// MPS_PREC_BF16X3, MPS_PREC_AUTO): the G1 step C = Q (B_q B_{q+1}) and the G3
// step B~_q = C V^dagger / ||s[:k]|| of the paper's Methods, "MPS algorithm
// for quantum circuit simulation" (Eqs. tildeC and Bl), on the TMA-fed
// tcgen05 GEMM of tc_tma.cuh.  Bond dimensions are read on the device, so the
// launches are sized for the bond capacities and capture into CUDA graphs.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include <cudaTypedefs.h>

#include "gate_kernels.cuh"
#include "internal.h"
#include "tc_tma.cuh"

namespace mpsv {

using namespace tma;

namespace {

// ---- theta: A = B_q as (2 chi_l) x chi_m, B = B_{q+1} as chi_m x (j, a_r)
struct ThetaSrcA {
  const float2* Bq;
  const int* chi;
  int q;
  __device__ void dims(int& rows, int& K) const {
    rows = 2 * chi[q];
    K = chi[q + 1];
  }
  __device__ float2 operator()(int r, int k) const { return Bq[(size_t)r * chi[q + 1] + k]; }
};

// Logical column n of a theta tile group: tile t = n / 64 holds a_r = 32 t ..
// 32 t + 31 for j = 0 (columns 0-31 of the tile) and j = 1 (32-63), so the
// epilogue finds both j of one a_r in one CTA.
struct ThetaSrcB {
  static constexpr bool kAlongN = true;  // consecutive a_r of one (k, j) are consecutive in memory
  const float2* Bq1;
  const int* chi;
  int q;
  __device__ void dims(int& npad, int& K) const {
    npad = (chi[q + 2] + 31) / 32 * 64;
    K = chi[q + 1];
  }
  __device__ float2 operator()(int k, int n, bool& ok) const {
    const int chi_r = chi[q + 2];
    const int w = n % 64, j = w / 32, ar = (n / 64) * 32 + (w % 32);
    ok = ar < chi_r;
    return ok ? Bq1[(size_t)(k * 2 + j) * chi_r + ar] : make_float2(0.f, 0.f);
  }
};

// out[(a_l, i), (j, a_r)] = sum_{i', j'} Q[2i + j][2i' + j'] acc[(a_l, i')][(j', a_r)],
// stored unscaled (the SVD kernel applies lam_q to its rows).  Output run h
// of a row is j = h: the 32 a_r of the tile at columns h chi_r + a_r.
struct ThetaEpi {
  const int* chi;
  int q;
  const DevGate* gate;
  float2* Cm;
  __device__ void dims(int& rows, int& kr, int& ncols) const {
    rows = 2 * chi[q];
    kr = 2 * chi[q + 1];
    ncols = (chi[q + 2] + 31) / 32 * 64;
  }
  __device__ void values(int row, int nbase, const float (&acc)[kBNr], float2 (&v)[64]) const {
    (void)nbase;
    const int i = row & 1;
    float2 g[2][4];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const double2 u = gate->u[(2 * i + j) * 4 + e];
        g[j][e] = make_float2(float(u.x), float(u.y));
      }
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      const float2 own0 = make_float2(acc[2 * c], acc[2 * c + 1]);
      const float2 own1 = make_float2(acc[64 + 2 * c], acc[64 + 2 * c + 1]);
      float2 oth0, oth1;  // the partner row (a_l, 1 - i)
      oth0.x = __shfl_xor_sync(0xffffffffu, own0.x, 1);
      oth0.y = __shfl_xor_sync(0xffffffffu, own0.y, 1);
      oth1.x = __shfl_xor_sync(0xffffffffu, own1.x, 1);
      oth1.y = __shfl_xor_sync(0xffffffffu, own1.y, 1);
      // value at (i', j'): i' == i -> own, else the partner's
      const float2 v00 = i == 0 ? own0 : oth0, v01 = i == 0 ? own1 : oth1;
      const float2 v10 = i == 1 ? own0 : oth0, v11 = i == 1 ? own1 : oth1;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        float2 o = make_float2(0.f, 0.f);
        cfma(o, g[j][0], v00);
        cfma(o, g[j][1], v01);
        cfma(o, g[j][2], v10);
        cfma(o, g[j][3], v11);
        v[32 * j + c] = o;
      }
    }
  }
  __device__ float2* run(int row, int nbase, int h, int& count) const {
    const int chi_r = chi[q + 2];
    const int ar0 = (nbase / 64) * 32;
    if (row >= 2 * chi[q] || ar0 >= chi_r) return nullptr;
    count = min(32, chi_r - ar0);
    return Cm + (size_t)row * (2 * chi_r) + h * chi_r + ar0;
  }
};

// ---- G3: A = C as (2 chi_l) x (2 chi_r), B(kk, a) = conj(B~_{q+1}[a][kk])
struct G3SrcA {
  const float2* Cm;
  const int* chi;
  int q;
  __device__ void dims(int& rows, int& K) const {
    rows = 2 * chi[q];
    K = 2 * chi[q + 2];
  }
  __device__ float2 operator()(int r, int k) const { return Cm[(size_t)r * (2 * chi[q + 2]) + k]; }
};

struct G3SrcB {
  static constexpr bool kAlongN = false;  // consecutive kk of one a are consecutive in memory
  const float2* Bn;
  const int* chi;
  int q;
  __device__ void dims(int& npad, int& K) const {
    npad = (chi[q + 1] + 63) / 64 * 64;
    K = 2 * chi[q + 2];
  }
  __device__ float2 operator()(int kk, int a, bool& ok) const {
    ok = a < chi[q + 1];
    if (!ok) return make_float2(0.f, 0.f);
    const float2 v = Bn[(size_t)a * (2 * chi[q + 2]) + kk];
    return make_float2(v.x, -v.y);
  }
};

struct G3Epi {
  const int* chi;
  int q;
  const DevReport* rep;
  float2* Bout;
  __device__ void dims(int& rows, int& kr, int& ncols) const {
    rows = 2 * chi[q];
    kr = 4 * chi[q + 2];
    ncols = (chi[q + 1] + 63) / 64 * 64;
  }
  __device__ void values(int row, int nbase, const float (&acc)[kBNr], float2 (&v)[64]) const {
    (void)row;
    (void)nbase;
    const float inv = float(rep->inv_norm);
#pragma unroll
    for (int c = 0; c < kBNc; ++c) v[c] = make_float2(acc[2 * c] * inv, acc[2 * c + 1] * inv);
  }
  // run h: new bond indices nbase + 32 h ..
  __device__ float2* run(int row, int nbase, int h, int& count) const {
    const int k = chi[q + 1], a0 = nbase + 32 * h;
    if (row >= 2 * chi[q] || a0 >= k) return nullptr;
    count = min(32, k - a0);
    return Bout + (size_t)row * k + a0;
  }
};

template <int M> CUtensorMapDataType map_type() {
  return M == kTF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
}

// The driver's tensor-map encoder, looked up through the runtime so that the
// library does not link the driver library itself (it loads on hosts without
// a GPU driver, where every entry point then fails cleanly).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag f;
  std::call_once(f, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

mps_status encode_map(CUtensorMap* map, CUtensorMapDataType type, void* base, uint64_t rows, uint64_t ld,
                      size_t elem) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available from the CUDA driver");
    return MPS_ECUDA;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld * elem)};
  const cuuint32_t box[2] = {(cuuint32_t)(kChunkBytes / elem), (cuuint32_t)kBM};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, type, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (%llu x %llu, %zu-byte elements) failed with CUresult %d",
              (unsigned long long)rows, (unsigned long long)ld, elem, (int)r);
    return MPS_ECUDA;
  }
  return MPS_OK;
}

template <int M> void set_attrs() {
  static std::once_flag f;
  std::call_once(f, [] {
    cudaFuncSetAttribute(cgemm_tma_kernel<M, ThetaEpi>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    cudaFuncSetAttribute(cgemm_tma_kernel<M, G3Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  });
}

// The GEMM over a grid of (column tiles, row tiles).
template <int M, class Epi>
void launch_gemm(const TcWork& w, dim3 grid, const Epi& epi, int* err, cudaStream_t s) {
  cgemm_tma_kernel<M, Epi><<<grid, kThreads, kSmemBytes, s>>>(w.maps[0], w.maps[1], w.maps[2], w.maps[3], epi, err);
}

// Blocks of 256 threads for `items` work items (grid-stride beyond 152 x 16 blocks).
int split_blocks(size_t items) { return (int)std::max<size_t>(1, std::min<size_t>((items + 255) / 256, 152 * 16)); }

// The two launches of the theta contraction for bond capacities (cap_l,
// cap_m, cap_r) around sites (q, q+1); the actual dimensions are chi[q..q+2].
template <int M>
void launch_theta_raw(const TcWork& w, const float2* Bq, const float2* Bq1, const int* chi, int q, int cap_l,
                      int cap_m, int cap_r, const DevGate* g, float2* Cm, int* err, cudaStream_t s) {
  using T = typename ModeTraits<M>::T;
  T* p[4];
  for (int i = 0; i < 4; ++i) p[i] = static_cast<T*>(w.planes[i]);
  const int npad_cap = (cap_r + 31) / 32 * 64, kpad_cap = pad_k(2 * cap_m, M) / 2;
  const int a_blocks = split_blocks((size_t)2 * cap_l * kpad_cap / 2);
  const int b_tiles = ((npad_cap + kSplitTile - 1) / kSplitTile) * ((kpad_cap + kSplitTile - 1) / kSplitTile);
  split_ab_kernel<M><<<a_blocks + std::min(b_tiles, 152 * 16), 256, 0, s>>>(
      ThetaSrcA{Bq, chi, q}, ThetaSrcB{Bq1, chi, q}, w.ld, a_blocks, p[0], p[1], p[2], p[3]);
  launch_gemm<M>(w, dim3(npad_cap / kBNc, (2 * cap_l + kBM - 1) / kBM), ThetaEpi{chi, q, g, Cm}, err, s);
}

template <int M>
void launch_theta(mps_state* st, const DevGate* g, int q, cudaStream_t s) {
  const float2* Bq = reinterpret_cast<const float2*>(st->d_B) + st->site_off[q];
  const float2* Bq1 = reinterpret_cast<const float2*>(st->d_B) + st->site_off[q + 1];
  KernelScope k(st->ctx, MPS_K_THETA);
  launch_theta_raw<M>(*st->tcw, Bq, Bq1, st->d_chi, q, st->cap[q], st->cap[q + 1], st->cap[q + 2], g,
                      reinterpret_cast<float2*>(st->d_C), &st->d_rep->tc_error, s);
}

template <int M>
void launch_g3(mps_state* st, int q, cudaStream_t s) {
  using T = typename ModeTraits<M>::T;
  TcWork& w = *st->tcw;
  const float2* Bn = reinterpret_cast<const float2*>(st->d_B) + st->site_off[q + 1];
  float2* Bout = reinterpret_cast<float2*>(st->d_B) + st->site_off[q];
  const int cap_l = st->cap[q], cap_m = st->cap[q + 1], cap_r = st->cap[q + 2];
  T* p[4];
  for (int i = 0; i < 4; ++i) p[i] = static_cast<T*>(w.planes[i]);
  KernelScope k(st->ctx, MPS_K_G3);
  const int npad_cap = (cap_m + 63) / 64 * 64, kpad_cap = pad_k(4 * cap_r, M) / 2;
  const int a_blocks = split_blocks((size_t)2 * cap_l * kpad_cap / 2);
  const int b_blocks = split_blocks((size_t)npad_cap * kpad_cap / 2);
  split_ab_kernel<M><<<a_blocks + b_blocks, 256, 0, s>>>(
      G3SrcA{reinterpret_cast<const float2*>(st->d_C), st->d_chi, q}, G3SrcB{Bn, st->d_chi, q}, w.ld, a_blocks, p[0],
      p[1], p[2], p[3]);
  launch_gemm<M>(w, dim3(npad_cap / kBNc, (2 * cap_l + kBM - 1) / kBM), G3Epi{st->d_chi, q, st->d_rep, Bout},
                 &st->d_rep->tc_error, s);
}

}  // namespace

// Planes and tensor maps for bond capacities up to maxcap in one mode.
static mps_status tc_work_alloc(mps_ctx* ctx, int maxcap, int mode, TcWork* w) {
  const size_t elem = mode == kTF32 ? 4 : 2;
  w->ld = pad_k(4 * maxcap, mode);                         // real K of both contractions (G3: 2 x 2 chi_r)
  w->rows_a = (2 * maxcap + kBM - 1) / kBM * kBM;          // 2 chi_l
  w->rows_b = 2 * ((maxcap + 31) / 32 * 64);               // embedded logical columns of theta (the larger)
  const size_t bytes_a = (size_t)w->rows_a * w->ld * elem, bytes_b = (size_t)w->rows_b * w->ld * elem;
  mps_status rc = MPS_OK;
  for (int i = 0; i < 4 && rc == MPS_OK; ++i) rc = dev_alloc(ctx, &w->planes[i], i < 2 ? bytes_a : bytes_b);
  const CUtensorMapDataType ty = mode == kTF32 ? map_type<kTF32>() : map_type<kBF16>();
  for (int i = 0; i < 4 && rc == MPS_OK; ++i)
    rc = encode_map(&w->maps[i], ty, w->planes[i], i < 2 ? w->rows_a : w->rows_b, w->ld, elem);
  if (rc == MPS_OK) {
    if (mode == kTF32)
      set_attrs<kTF32>();
    else
      set_attrs<kBF16>();
  }
  return rc;
}

static void tc_work_free(mps_ctx* ctx, TcWork* w) {
  if (!w) return;
  for (void*& p : w->planes) {
    dev_free(ctx, p);
    p = nullptr;
  }
}

mps_status tc_gates_setup(mps_state* st) {
  int maxcap = 1;
  for (int c : st->cap) maxcap = std::max(maxcap, c);
  st->tcw = new TcWork();  // freed by tc_gates_free whatever happens
  return tc_work_alloc(st->ctx, maxcap, st->tc_gates == MPS_PREC_BF16X3 ? kBF16 : kTF32, st->tcw);
}

void tc_gates_free(mps_state* st) {
  if (!st->tcw) return;
  tc_work_free(st->ctx, st->tcw);
  delete st->tcw;
  st->tcw = nullptr;
}

bool tc_gates_used(const mps_state* st, int q) {
  if (!st->tcw) return false;
  // AUTO keeps small contractions on the CUDA cores: the 128 x 64 tiles only pay off at large bond dimensions
  const int min_cap = st->tc_gates == MPS_PREC_AUTO ? 256 : 32;
  return std::max(st->cap[q], st->cap[q + 2]) >= min_cap;
}

void tc_theta(mps_state* st, const DevGate* g, int q, cudaStream_t s) {
  if (st->tc_gates == MPS_PREC_BF16X3)
    launch_theta<kBF16>(st, g, q, s);
  else
    launch_theta<kTF32>(st, g, q, s);
}

void tc_g3(mps_state* st, int q, cudaStream_t s) {
  if (st->tc_gates == MPS_PREC_BF16X3)
    launch_g3<kBF16>(st, q, s);
  else
    launch_g3<kTF32>(st, q, s);
}

// Workspace of mps_contract_theta, kept by its context and grown on demand.
struct ContractWork {
  int mode = -1, cap = 0;
  TcWork tcw;
  int* d_chi = nullptr;
  DevGate* d_gate = nullptr;
  double* d_ones = nullptr;
  DevReport* d_rep = nullptr;
};

void contract_work_free(mps_ctx* ctx) {
  if (!ctx->contract) return;
  ContractWork* c = ctx->contract;
  tc_work_free(ctx, &c->tcw);
  for (void* p : {(void*)c->d_chi, (void*)c->d_gate, (void*)c->d_ones, (void*)c->d_rep}) dev_free(ctx, p);
  delete c;
  ctx->contract = nullptr;
}

}  // namespace mpsv

using namespace mpsv;

extern "C" mps_status mps_contract_theta(mps_ctx* ctx, int32_t precision, int32_t chi_l, int32_t chi_m,
                                         int32_t chi_r, const void* B_left, const void* B_right, const double* gate,
                                         void* C_out) {
  if (!ctx || !B_left || !B_right || !gate || !C_out) {
    set_error("mps_contract_theta: NULL argument");
    return MPS_EINVAL;
  }
  if (precision != MPS_PREC_FP32 && precision != MPS_PREC_TF32X3 && precision != MPS_PREC_BF16X3) {
    set_error("mps_contract_theta: precision %d is not MPS_PREC_FP32, MPS_PREC_TF32X3 or MPS_PREC_BF16X3", precision);
    return MPS_EINVAL;
  }
  if (chi_l < 1 || chi_m < 1 || chi_r < 1 || chi_l > 4096 || chi_m > 4096 || chi_r > 4096) {
    set_error("mps_contract_theta: bond dimensions (%d, %d, %d) outside 1..4096", chi_l, chi_m, chi_r);
    return MPS_EINVAL;
  }
  DeviceGuard guard(ctx->device);
  cudaStream_t s = ctx->stream;
  const int cap = std::max(chi_l, std::max(chi_m, chi_r));
  const int mode = precision == MPS_PREC_BF16X3 ? kBF16 : kTF32;
  ContractWork* c = ctx->contract;
  const bool need_tc = precision != MPS_PREC_FP32;
  if (c && (cap > c->cap || (need_tc && c->mode != mode))) {
    MPSV_CUDA(cudaStreamSynchronize(s));  // the old workspace may still be read
    contract_work_free(ctx);
    c = nullptr;
  }
  if (!c) {
    c = new ContractWork();
    ctx->contract = c;
    c->cap = cap;
    c->mode = need_tc ? mode : -1;
    mps_status rc = dev_alloc(ctx, (void**)&c->d_chi, 4 * sizeof(int));
    if (rc == MPS_OK) rc = dev_alloc(ctx, (void**)&c->d_gate, sizeof(DevGate));
    if (rc == MPS_OK) rc = dev_alloc(ctx, (void**)&c->d_rep, sizeof(DevReport));
    if (rc == MPS_OK) rc = dev_alloc(ctx, (void**)&c->d_ones, (size_t)cap * sizeof(double));
    if (rc == MPS_OK && need_tc) rc = tc_work_alloc(ctx, cap, mode, &c->tcw);
    if (rc == MPS_OK) {
      std::vector<double> ones(cap, 1.0);
      cudaError_t e = cudaMemcpyAsync(c->d_ones, ones.data(), cap * sizeof(double), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(c->d_rep, 0, sizeof(DevReport), s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) rc = cuda_fail(e, "mps_contract_theta set-up");
    }
    if (rc != MPS_OK) {
      contract_work_free(ctx);
      return rc;
    }
  }
  DevGate hg;
  std::memset(&hg, 0, sizeof(hg));
  hg.arity = 2;
  for (int e = 0; e < 16; ++e) hg.u[e] = make_double2(gate[2 * e], gate[2 * e + 1]);
  const int hchi[4] = {chi_l, chi_m, chi_r, 0};
  // stream-ordered uploads from pageable host memory: the copies are staged
  // before the call returns, so the host arrays may change afterwards
  MPSV_CUDA(cudaMemcpyAsync(c->d_gate, &hg, sizeof(DevGate), cudaMemcpyHostToDevice, s));
  MPSV_CUDA(cudaMemcpyAsync(c->d_chi, hchi, sizeof(hchi), cudaMemcpyHostToDevice, s));
  const float2* Bq = static_cast<const float2*>(B_left);
  const float2* Bq1 = static_cast<const float2*>(B_right);
  float2* Cm = static_cast<float2*>(C_out);
  {
    KernelScope k(ctx, MPS_K_THETA);
    if (!need_tc) {
      const dim3 blk(kTile, kTile), grid((chi_r + kTile - 1) / kTile, (chi_l + kTile - 1) / kTile);
      theta_kernel<float, float><<<grid, blk, 0, s>>>(Bq, Bq1, c->d_gate, c->d_ones, c->d_chi, 0, Cm,
                                                      (float2*)nullptr);
    } else if (mode == kTF32) {
      launch_theta_raw<kTF32>(c->tcw, Bq, Bq1, c->d_chi, 0, chi_l, chi_m, chi_r, c->d_gate, Cm, &c->d_rep->tc_error,
                              s);
    } else {
      launch_theta_raw<kBF16>(c->tcw, Bq, Bq1, c->d_chi, 0, chi_l, chi_m, chi_r, c->d_gate, Cm, &c->d_rep->tc_error,
                              s);
    }
  }
  MPSV_CUDA(cudaGetLastError());
  return MPS_OK;
}
