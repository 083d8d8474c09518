// mps_gate2_noalloc: one two-qubit gate on caller-owned device buffers, with
// no device allocation at all.
//
// The regular path keeps its gate scratch (the theta product C, the Jacobi
// matrices A and V, the bond dimensions and the truncation report) in
// per-state buffers from cudaMalloc.  Some callers cannot allocate: code
// running inside a CUDA host callback or stream-ordered host function (where
// CUDA API calls that allocate are not allowed), embedders that hand the
// library a fixed, pre-partitioned slice of device memory, or processes whose
// memory budget was fixed when they started.  For them this entry point
// takes its scratch from a file-scope __device__ array of fixed size,
// kMaxBytes below.  That array is part of the library image: every GPU that
// loads libmpsvqe.so holds it until the process exits.
//
// Host code cannot use the array's name as a device address (on the host it
// is only a stand-in symbol), so the first call on each device, with that
// device current, asks the runtime for the address with cudaGetSymbolAddress
// and keeps it.  Make that first call before capturing a stream into a CUDA
// graph.
//
// All calls share the one array and it keeps the last call's contents: the
// kernels overwrite everything they read, and calls whose work overlaps on
// the GPU (other streams, other host threads) race on it.
#include <mutex>

#include "gate_kernels.cuh"
#include "internal.h"

namespace mpsv {
namespace {

constexpr int kMaxChi = 32;                 // largest chi_l, chi_r accepted
constexpr int kMaxDim = 2 * kMaxChi;        // theta is at most 64 x 64
constexpr size_t kMatBytes = (size_t)kMaxDim * kMaxDim * sizeof(double2);
constexpr size_t kOffC = 0, kOffA = kMatBytes, kOffV = 2 * kMatBytes;
constexpr size_t kOffChi = 3 * kMatBytes;                 // int[4]
constexpr size_t kOffGate = kOffChi + 256;                // DevGate
constexpr size_t kOffRep = kOffGate + 512;                // DevReport
constexpr size_t kMaxBytes = kOffRep + 256;               // 197,632 bytes

__device__ __align__(256) unsigned char g_noalloc_scratch[kMaxBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {};

// Per-device set-up: the scratch address and the SVD kernel's shared-memory limit.
mps_status scratch_for(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("mps_gate2_noalloc: device %d outside 0..%d", dev, kMaxDevices - 1);
    return MPS_EINVAL;
  }
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "mps_gate2_noalloc: cudaGetSymbolAddress");
    int smem = 0;
    e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(svd_truncate_kernel<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               smem - 1024);
    if (e != cudaSuccess) return cuda_fail(e, "mps_gate2_noalloc: set-up");
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return MPS_OK;
}

// Writes the bond dimensions and the gate into the scratch and clears the report.
__global__ void noalloc_setup_kernel(unsigned char* scratch, int chi_l, int chi_m, int chi_r, DevGate g) {
  int* chi = reinterpret_cast<int*>(scratch + kOffChi);
  if (threadIdx.x == 0) {
    chi[0] = chi_l;
    chi[1] = chi_m;
    chi[2] = chi_r;
    DevReport* r = reinterpret_cast<DevReport*>(scratch + kOffRep);
    r->discarded_weight = 0.0;
    r->min_kept_sv = 1.0;
    r->inv_norm = 1.0;
    r->max_chi = 1;
    r->degenerate_cuts = 0;
    r->not_converged = 0;
    r->max_sweeps = 0;
    r->two_qubit_gates = 0;
    r->svd_flops = 0.0;
    r->tc_error = 0;
    r->sweeps_fp32 = r->sweeps_fp64 = 0;
    for (int i = 0; i < 4; ++i) r->phase_cycles[i] = 0.0;
  }
  DevGate* d = reinterpret_cast<DevGate*>(scratch + kOffGate);
  if (threadIdx.x < 16) d->u[threadIdx.x] = g.u[threadIdx.x];
  if (threadIdx.x == 0) {
    d->q = 0;
    d->arity = 2;
  }
}

__global__ void noalloc_finish_kernel(const unsigned char* scratch, int* chi_out) {
  if (threadIdx.x == 0) *chi_out = reinterpret_cast<const int*>(scratch + kOffChi)[1];
}

}  // namespace
}  // namespace mpsv

using namespace mpsv;

extern "C" mps_status mps_gate2_noalloc(int device, void* cuda_stream, int32_t chi_l, int32_t chi_m, int32_t chi_r,
                                        double* B_left, double* B_right, const double* lam_left, double* lam_out,
                                        const double* gate, int32_t chi_max, double trunc_rel,
                                        int32_t* chi_out) {
  if (!B_left || !B_right || !lam_left || !lam_out || !gate || !chi_out) {
    set_error("mps_gate2_noalloc: NULL argument");
    return MPS_EINVAL;
  }
  if (chi_l < 1 || chi_m < 1 || chi_r < 1 || chi_l > kMaxChi || chi_r > kMaxChi || chi_m > 2 * kMaxChi) {
    set_error("mps_gate2_noalloc: bond dimensions (%d, %d, %d) outside 1..%d (chi_l, chi_r) and 1..%d (chi_m); "
              "the fixed scratch holds a theta of at most %d x %d",
              chi_l, chi_m, chi_r, kMaxChi, 2 * kMaxChi, kMaxDim, kMaxDim);
    return MPS_EINVAL;
  }
  if (chi_max < 1 || !(trunc_rel >= 0.0 && trunc_rel < 1.0)) {
    set_error("mps_gate2_noalloc: chi_max = %d, trunc_rel = %g", chi_max, trunc_rel);
    return MPS_EINVAL;
  }
  int count = 0;
  cudaError_t ce = cudaGetDeviceCount(&count);
  if (ce != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    set_error("mps_gate2_noalloc: no CUDA device %d (%d visible)", device, ce == cudaSuccess ? count : 0);
    return ce != cudaSuccess ? MPS_ECUDA : MPS_EINVAL;
  }
  int prev = -1;
  ce = cudaGetDevice(&prev);
  if (ce == cudaSuccess && prev != device) ce = cudaSetDevice(device);
  if (ce != cudaSuccess) return cuda_fail(ce, "mps_gate2_noalloc: cudaSetDevice");
  struct Restore {
    int prev, dev;
    ~Restore() {
      if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    }
  } restore{prev, device};
  unsigned char* scratch = nullptr;
  mps_status rc = scratch_for(device, &scratch);
  if (rc != MPS_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  DevGate g;
  for (int e = 0; e < 16; ++e) g.u[e] = make_double2(gate[2 * e], gate[2 * e + 1]);
  g.q = 0;
  g.arity = 2;
  noalloc_setup_kernel<<<1, 32, 0, s>>>(scratch, chi_l, chi_m, chi_r, g);
  int* chi = reinterpret_cast<int*>(scratch + kOffChi);
  const DevGate* dg = reinterpret_cast<const DevGate*>(scratch + kOffGate);
  DevReport* rep = reinterpret_cast<DevReport*>(scratch + kOffRep);
  double2* C = reinterpret_cast<double2*>(scratch + kOffC);
  double2* A = reinterpret_cast<double2*>(scratch + kOffA);
  double2* V = reinterpret_cast<double2*>(scratch + kOffV);
  double2* Bl = reinterpret_cast<double2*>(B_left);
  double2* Br = reinterpret_cast<double2*>(B_right);
  const dim3 blk(kTile, kTile);
  theta_kernel<double, double><<<dim3((chi_r + kTile - 1) / kTile, (chi_l + kTile - 1) / kTile), blk, 0, s>>>(
      Bl, Br, dg, lam_left, chi, 0, C, A);
  SvdParams p;
  p.chi_max = chi_max;
  p.max_sweeps = 60;
  p.trunc_rel = trunc_rel;
  p.tol = 0.0;
  p.mixed = 0;
  const int n = 2 * chi_r, m = 2 * chi_l;
  const size_t smem = ((size_t)m * n + (size_t)n * n) * sizeof(double2) + (size_t)n * (sizeof(double) + sizeof(int)) + 64;
  svd_truncate_kernel<double, double><<<1, 32 * std::min(32, std::max(1, n / 2)), smem, s>>>(
      A, V, 1, chi, 0, p, Br, lam_out, rep);
  const int kmax = std::min(chi_max, std::min(m, n));
  g3_kernel<double><<<dim3((kmax + kTile - 1) / kTile, (m + kTile - 1) / kTile), blk, 0, s>>>(C, Br, chi, 0, rep, Bl);
  noalloc_finish_kernel<<<1, 32, 0, s>>>(scratch, chi_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "mps_gate2_noalloc launch");
  return MPS_OK;
}
