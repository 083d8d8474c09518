// Host-side objects behind the opaque handles of mps_vqe.h.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "../../include/mps_vqe.h"
#include "common.cuh"

namespace mpsv {

void set_error(const char* fmt, ...);
mps_status cuda_fail(cudaError_t e, const char* what);
const char* last_error();

#define MPSV_CUDA(call)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// A circuit's bind + gate launches captured once for one state and replayed
// as a CUDA graph.  Kernel timing inside the graph uses events owned by the
// graph (re-recorded by every replay).
struct CircuitGraph {
  uint64_t circ_serial = 0;
  const void* theta_ptr = nullptr;
  const void* bound_ptr = nullptr;
  uint32_t mask = 0;
  cudaGraphExec_t exec = nullptr;
  struct Timing {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Timing> timing;
  long long counts[MPS_K_COUNT] = {};  // launches per replay
  long long unread = 0;                // replays since the last profile collection
};

}  // namespace mpsv

namespace mpsv {
struct ContractWork;
void contract_work_free(mps_ctx* ctx);
struct SvdWork;
void svd_work_free(mps_ctx* ctx);
}  // namespace mpsv

struct mps_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t alloc_limit = 0;
  size_t allocated = 0;
  std::map<void*, size_t> allocs;
  // kernel accounting (mps_ctx_profile)
  uint32_t prof_mask = 0;
  long long launches[MPS_K_COUNT] = {};
  long long timed[MPS_K_COUNT] = {};
  double ms[MPS_K_COUNT] = {};
  struct Pending {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  bool use_graphs = true;                           // replay circuits as CUDA graphs (mps_ctx_set_graphs)
  mpsv::CircuitGraph* capturing = nullptr;          // graph being captured on this context's stream
  mpsv::ContractWork* contract = nullptr;           // workspace of mps_contract_theta
  mpsv::SvdWork* svdw = nullptr;                     // workspace of mps_truncated_svd
  std::vector<mpsv::CircuitGraph*> graph_watch;     // graphs replayed since the last profile collection
};

namespace mpsv {
// Bracket one kernel launch for accounting: KernelScope k(ctx, kind); launch<<<...>>>;
struct KernelScope {
  mps_ctx* c;
  int kind;
  cudaEvent_t a = nullptr, b = nullptr;
  KernelScope(mps_ctx* ctx, int k);
  ~KernelScope();
};
}  // namespace mpsv

namespace mpsv {
mps_status dev_alloc(mps_ctx* ctx, void** p, size_t bytes);
void dev_free(mps_ctx* ctx, void* p);
}  // namespace mpsv

namespace mpsv {
// Workspace of the tensor-core gate contractions (tc_gates.cu): the hi / lo
// operand planes (A_hi, A_lo, B_hi, B_lo; K-major, ld elements per row) and
// their TMA tensor maps, sized once for the state's largest bond capacity.
struct TcWork {
  void* planes[4] = {nullptr, nullptr, nullptr, nullptr};
  CUtensorMap maps[4];
  int ld = 0, rows_a = 0, rows_b = 0;
};
}  // namespace mpsv

struct mps_state {
  mps_ctx* ctx = nullptr;
  int n = 0;
  mps_config cfg{};
  bool fp32 = false;   // complex64 storage
  bool svd64 = true;   // FP64 Jacobi
  bool tc = false;     // tensor-core environment contractions (complex64 states)
  std::vector<int> cap;          // bond capacities, n + 1
  std::vector<size_t> site_off;  // complex elements
  std::vector<size_t> lam_off;   // doubles
  void* d_B = nullptr;
  double* d_lam = nullptr;
  int* d_chi = nullptr;
  size_t* d_site_off = nullptr;
  size_t* d_lam_off = nullptr;
  uint8_t* d_bits = nullptr;
  mpsv::DevReport* d_rep = nullptr;
  void* d_C = nullptr;  // theta C, m x n (storage precision)
  void* d_A = nullptr;  // SVD matrix, m x n (SVD precision)
  void* d_V = nullptr;  // n x n (SVD precision)
  mpsv::DevGate* d_gates = nullptr;
  size_t gates_cap = 0;
  size_t total_lam = 0;
  size_t total_elems = 0;
  std::vector<uint8_t> last_bits;
  bool broken = false;
  int nc_seen = 0;  // svd_not_converged as last read by the host (mps_apply_gates)
  // split-product tensor-core gate contractions: 0 (CUDA cores) or the
  // mps_precision that selected them (TF32X3, BF16X3, AUTO)
  int tc_gates = 0;
  mpsv::TcWork* tcw = nullptr;
  // circuit binding workspace (per state, so states sharing a circuit can run concurrently)
  mpsv::DevGate* d_bound = nullptr;
  size_t bound_cap = 0;
  double* d_theta = nullptr;
  size_t theta_cap = 0;
  // energy workspace (per state, so states sharing a Hamiltonian can run concurrently)
  void* d_L[2] = {nullptr, nullptr};
  void* d_M = nullptr;
  size_t L_bytes = 0, M_bytes = 0;
  double* d_vals = nullptr;
  size_t vals_cap = 0;
  double* d_energy = nullptr;
  mpsv::CircuitGraph* graph = nullptr;  // last captured circuit (graph replay)
  // linear observables over per-string expectations (mps_observables_eval)
  double2* d_obs = nullptr;
  size_t obs_cap = 0;
};

struct mps_circuit {
  mps_ctx* ctx = nullptr;
  uint64_t serial = 0;  // unique per created circuit (graph cache key)
  int n = 0;
  int n_params = 0;
  int n_gates = 0;
  std::vector<int> q, arity;
  mpsv::DevTmplGate* d_tmpl = nullptr;
};

namespace mpsv {
struct LevelHost {
  int n_parents = 0, n_children = 0, n_leaves = 0, n_traces = 0;
  size_t off_parent = 0, off_child = 0, off_leaf = 0, off_trace = 0;
  int n_dense = 0, n_diag = 0;  // parents with a stored environment / starting strings here
  size_t off_dense = 0, off_diag = 0;
};
}  // namespace mpsv

struct mps_ham {
  mps_ctx* ctx = nullptr;
  int n = 0;
  long long n_terms = 0;
  long long n_nodes = 0;
  long long max_level_nodes = 0;
  std::vector<mpsv::LevelHost> levels;
  int* d_parent_src = nullptr;
  int2* d_child = nullptr;
  int4* d_leaf = nullptr;
  int2* d_trace = nullptr;
  int2* d_dense = nullptr;  // (parent entry, environment slot)
  int* d_diag = nullptr;    // parent entry
  double* d_coeffs = nullptr;
};

namespace mpsv {
// The two status flags of a state, read back with one 8-byte copy from
// &DevReport::not_converged.
struct StateFlags {
  int not_converged;  // SVDs that reached the sweep cap since the last reset
  int tc_error;       // a tensor-core kernel ran out of its bounded wait
};
static_assert(offsetof(DevReport, tc_error) == offsetof(DevReport, not_converged) + sizeof(int),
              "StateFlags mirrors two adjacent DevReport fields");
// Queues the read of a state's flags into *f (valid once the stream has synchronised).
cudaError_t queue_flags(mps_state* st, StateFlags* f);
// The status an evaluation reports for its flags: MPS_ETIMEOUT for a
// tensor-core timeout, else MPS_ENOTCONV when gates count and an SVD reached
// its sweep cap (the results are written as they stand), else MPS_OK.
mps_status flags_status(const StateFlags& f, bool gates);
// A status that still delivers its result (the energy, the updated state).
inline bool status_has_result(mps_status s) { return s == MPS_OK || s == MPS_ENOTCONV; }

// state.cu
mps_status state_apply_device_gates(mps_state* st, const DevGate* d_gates, const int* q, const int* arity, size_t n);
mps_status state_reset(mps_state* st, const uint8_t* bits);
// Copies theta into the state's workspace and binds the circuit's gates there.
mps_status state_bind_circuit(mps_state* st, const mps_circuit* c, const double* theta, int theta_on_device);
// Binds theta and applies the whole circuit: a CUDA graph captured on first
// use for this (state, circuit) and replayed afterwards.
mps_status state_run_circuit(mps_state* st, const mps_circuit* c, const double* theta, int theta_on_device);
void graph_destroy(mps_ctx* ctx, CircuitGraph* g);
// energy.cu
mps_status ham_energy_async(mps_state* st, mps_ham* h, double* d_out);
// tc_gates.cu
mps_status tc_gates_setup(mps_state* st);
void tc_gates_free(mps_state* st);
bool tc_gates_used(const mps_state* st, int q);  // this bond's gates take the tensor-core contractions
void tc_theta(mps_state* st, const DevGate* g, int q, cudaStream_t s);
void tc_g3(mps_state* st, int q, cudaStream_t s);
}  // namespace mpsv
