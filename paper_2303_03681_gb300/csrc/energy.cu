// Hamiltonian upload (prefix trie of the Pauli strings) and the Pauli-sum
// energy of Eq. expec2 with shared left environments.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>

#include "gate_kernels.cuh"
#include "energy_kernels.cuh"
#include "internal.h"
#include "tc_gemm.cuh"

namespace mpsv {

namespace {

struct Node {
  int level;   // site of the last operator; -1 for a start node
  int parent;  // node id; start nodes have -1
  int op;
  int slot = -1;   // environment slot at its level (nodes with children)
  int entry = -1;  // parent-entry index at the next level (nodes with children, start nodes)
  bool has_child = false;
  std::vector<int> terms;
};

}  // namespace

// Builds the trie on the host.  Start node s (id s < n) stands for diag(lam_s^2)
// on the bond left of site s; node (parent, op) extends its parent's string by
// one site.
static mps_status build_trie(mps_ham* h, const uint8_t* ops, const double* coeffs, std::vector<int>& parent_src,
                             std::vector<int2>& child, std::vector<int4>& leaf, std::vector<int2>& trace,
                             std::vector<int2>& dense, std::vector<int>& diag) {
  const int n = h->n;
  std::vector<Node> nodes(n);
  for (int s = 0; s < n; ++s) {
    nodes[s].level = -1;
    nodes[s].parent = -1;
    nodes[s].op = 0;
  }
  std::unordered_map<uint64_t, int> edge;
  edge.reserve(1 << 16);
  for (long long t = 0; t < h->n_terms; ++t) {
    const uint8_t* row = ops + (size_t)t * n;
    int first = -1, last = -1;
    for (int j = 0; j < n; ++j) {
      if (row[j] > 3) {
        set_error("mps_hamiltonian_create: ops[%lld, %d] = %d is not in 0..3", t, j, (int)row[j]);
        return MPS_EINVAL;
      }
      if (row[j]) {
        if (first < 0) first = j;
        last = j;
      }
    }
    if (!std::isfinite(coeffs[t])) {
      set_error("mps_hamiltonian_create: coefficient %lld is not finite", t);
      return MPS_EINVAL;
    }
    if (first < 0) continue;  // identity: <I> = 1 (vals prefilled)
    int cur = first;
    for (int j = first; j <= last; ++j) {
      const uint64_t key = ((uint64_t)cur << 2) | row[j];
      auto it = edge.find(key);
      int nxt;
      if (it == edge.end()) {
        nxt = (int)nodes.size();
        Node nd;
        nd.level = j;
        nd.parent = cur;
        nd.op = row[j];
        nodes.push_back(nd);
        edge.emplace(key, nxt);
      } else {
        nxt = it->second;
      }
      nodes[cur].has_child = true;
      cur = nxt;
    }
    nodes[cur].terms.push_back((int)t);
  }
  // bucket real nodes by level (creation order inside a level)
  std::vector<std::vector<int>> by_level(n);
  for (size_t id = n; id < nodes.size(); ++id) by_level[nodes[id].level].push_back((int)id);
  h->levels.assign(n, LevelHost());
  long long n_mat = 0, max_level = 0;
  for (int j = 0; j < n; ++j) {
    LevelHost& L = h->levels[j];
    L.off_parent = parent_src.size();
    L.off_child = child.size();
    L.off_leaf = leaf.size();
    L.off_trace = trace.size();
    int n_entries = 0;
    int slots = 0;
    for (int id : by_level[j]) {
      Node& nd = nodes[id];
      Node& par = nodes[nd.parent];
      if (par.entry < 0) {
        par.entry = n_entries++;
        parent_src.push_back(par.level < 0 ? -1 : par.slot);
      }
      if (nd.has_child) {
        nd.slot = slots++;
        child.push_back(make_int2(par.entry, nd.op));
      }
    }
    for (int id : by_level[j]) {
      const Node& nd = nodes[id];
      for (int t : nd.terms) {
        if (nd.has_child)
          trace.push_back(make_int2(nd.slot, t));
        else
          leaf.push_back(make_int4(nodes[nd.parent].entry, nd.op, t, 0));
      }
    }
    L.off_dense = dense.size();
    L.off_diag = diag.size();
    for (int e = 0; e < n_entries; ++e) {
      const int src = parent_src[L.off_parent + e];
      if (src < 0)
        diag.push_back(e);
      else
        dense.push_back(make_int2(e, src));
    }
    L.n_dense = (int)(dense.size() - L.off_dense);
    L.n_diag = (int)(diag.size() - L.off_diag);
    L.n_parents = n_entries;
    L.n_children = slots;
    L.n_leaves = (int)(leaf.size() - L.off_leaf);
    L.n_traces = (int)(trace.size() - L.off_trace);
    n_mat += slots;
    max_level = std::max<long long>(max_level, slots);
  }
  h->n_nodes = n_mat;
  h->max_level_nodes = max_level;
  return MPS_OK;
}

// Environment buffers sized for the bond dimensions the state has now
// (grow-only); slot strides follow the same dimensions.
template <typename R>
static mps_status ensure_env_buffers(const std::vector<int>& chi, mps_state* st, const mps_ham* h) {
  size_t Lneed = 16, Mneed = 16;
  for (int j = 0; j < h->n; ++j) {
    const LevelHost& L = h->levels[j];
    const size_t cl = chi[j], cr = chi[j + 1];
    Lneed = std::max(Lneed, (size_t)L.n_children * cr * cr * sizeof(cplx<R>));
    Mneed = std::max(Mneed, (size_t)L.n_parents * 2 * cl * cr * sizeof(cplx<R>));
  }
  mps_ctx* c = st->ctx;
  if (Lneed > st->L_bytes) {
    dev_free(c, st->d_L[0]);
    dev_free(c, st->d_L[1]);
    st->d_L[0] = st->d_L[1] = nullptr;
    st->L_bytes = 0;
    mps_status rc = dev_alloc(c, &st->d_L[0], Lneed);
    if (rc == MPS_OK) rc = dev_alloc(c, &st->d_L[1], Lneed);
    if (rc != MPS_OK) return rc;
    st->L_bytes = Lneed;
  }
  if (Mneed > st->M_bytes) {
    dev_free(c, st->d_M);
    st->d_M = nullptr;
    st->M_bytes = 0;
    mps_status rc = dev_alloc(c, &st->d_M, Mneed);
    if (rc != MPS_OK) return rc;
    st->M_bytes = Mneed;
  }
  if ((size_t)h->n_terms > st->vals_cap || !st->d_vals) {
    dev_free(c, st->d_vals);
    st->d_vals = nullptr;
    st->vals_cap = 0;
    mps_status rc = dev_alloc(c, (void**)&st->d_vals, std::max<size_t>(16, h->n_terms * sizeof(double)));
    if (rc != MPS_OK) return rc;
    st->vals_cap = h->n_terms;
  }
  if (!st->d_energy) {
    mps_status rc = dev_alloc(c, (void**)&st->d_energy, sizeof(double));
    if (rc != MPS_OK) return rc;
  }
  return MPS_OK;
}

// Smallest bond dimension (either side of a site) whose environment
// contractions go to the tensor cores when a state allows them.
constexpr int kTcMinChi = 64;

// Tensor-core path of one level (complex64 only).  Returns false if a launch failed.
template <typename R>
static bool launch_env_tc(mps_state*, mps_ham*, const LevelHost&, int, const std::vector<int>&, const cplx<R>*,
                          const cplx<R>*, cplx<R>*, cplx<R>*) {
  return false;  // complex128 states never take this path
}

template <>
bool launch_env_tc<float>(mps_state* st, mps_ham* h, const LevelHost& L, int j, const std::vector<int>& chi,
                          const float2* Lprev, const float2* Bj, float2* M, float2* Lcur) {
  // the shared-memory opt-in is a per-device function attribute
  static std::mutex mu;
  static uint64_t done_mask = 0;
  mps_ctx* c = st->ctx;
  {
    std::lock_guard<std::mutex> g(mu);
    const uint64_t bit = 1ull << (c->device & 63);
    if (!(done_mask & bit)) {
      if (cudaFuncSetAttribute(tc::cgemm_kernel<EnvMProb>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)tc::kSmemBytes) != cudaSuccess ||
          cudaFuncSetAttribute(tc::cgemm_kernel<EnvChildProb>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)tc::kSmemBytes) != cudaSuccess)
        return false;
      done_mask |= bit;
    }
  }
  cudaStream_t s = c->stream;
  const int chi_l = chi[j], chi_r = chi[j + 1];
  int* err = &st->d_rep->tc_error;
  if (L.n_diag) {
    KernelScope k(c, MPS_K_ENV_M);
    const size_t tot = (size_t)L.n_diag * chi_l * 2 * chi_r;
    env_m_diag_kernel<float><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
        h->d_diag + L.off_diag, L.n_diag, Bj, st->d_lam + st->lam_off[j], chi_l, chi_r, M);
  }
  if (L.n_dense) {
    KernelScope k(c, MPS_K_ENV_M);
    EnvMProb p{h->d_dense + L.off_dense, Lprev, Bj, M, chi_l, chi_r};
    const int tiles_n = (2 * chi_r + tc::kBN / 2 - 1) / (tc::kBN / 2);
    const dim3 grid((unsigned)((size_t)L.n_dense * tiles_n), (unsigned)((chi_l + tc::kBM - 1) / tc::kBM));
    tc::cgemm_kernel<EnvMProb><<<grid, tc::kThreads, tc::kSmemBytes, s>>>(p, tiles_n, err);
  }
  if (L.n_children) {
    KernelScope k(c, MPS_K_ENV_CHILD);
    EnvChildProb p{h->d_child + L.off_child, Bj, M, Lcur, chi_l, chi_r};
    const int tiles_n = (chi_r + tc::kBN / 2 - 1) / (tc::kBN / 2);
    const dim3 grid((unsigned)((size_t)L.n_children * tiles_n), (unsigned)((chi_r + tc::kBM - 1) / tc::kBM));
    tc::cgemm_kernel<EnvChildProb><<<grid, tc::kThreads, tc::kSmemBytes, s>>>(p, tiles_n, err);
  }
  return cudaPeekAtLastError() == cudaSuccess;
}

template <typename R>
static mps_status energy_levels(mps_state* st, mps_ham* h, double* d_out) {
  cudaStream_t s = st->ctx->stream;
  // One read of the bond dimensions sizes every grid of this evaluation.
  std::vector<int> chi(st->n + 1);
  MPSV_CUDA(cudaMemcpyAsync(chi.data(), st->d_chi, (st->n + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
  MPSV_CUDA(cudaStreamSynchronize(s));
  for (int b = 0; b <= st->n; ++b) {
    if (chi[b] < 1 || chi[b] > st->cap[b]) {
      set_error("energy: bond %d has dimension %d outside 1..%d (state corrupted)", b, chi[b], st->cap[b]);
      st->broken = true;
      return MPS_ESTATE;
    }
  }
  mps_status rc = ensure_env_buffers<R>(chi, st, h);
  if (rc != MPS_OK) return rc;
  const long long nt = h->n_terms;
  mps_ctx* c = st->ctx;
  if (st->tc) MPSV_CUDA(cudaMemsetAsync(&st->d_rep->tc_error, 0, sizeof(int), s));
  if (nt) {
    KernelScope k(c, MPS_K_SETUP);
    fill_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(st->d_vals, nt, 1.0);
  }
  const cplx<R>* B = reinterpret_cast<const cplx<R>*>(st->d_B);
  cplx<R>* Lprev = reinterpret_cast<cplx<R>*>(st->d_L[0]);
  cplx<R>* Lcur = reinterpret_cast<cplx<R>*>(st->d_L[1]);
  cplx<R>* M = reinterpret_cast<cplx<R>*>(st->d_M);
  const dim3 blk(kTile, kTile);
  for (int j = 0; j < h->n; ++j) {
    const LevelHost& L = h->levels[j];
    if (!L.n_parents) continue;
    EnvLevel lv;
    lv.parent_src = h->d_parent_src + L.off_parent;
    lv.child = h->d_child + L.off_child;
    lv.leaf = h->d_leaf + L.off_leaf;
    lv.trace = h->d_trace + L.off_trace;
    lv.n_parents = L.n_parents;
    lv.n_children = L.n_children;
    lv.n_leaves = L.n_leaves;
    lv.n_traces = L.n_traces;
    lv.site = j;
    lv.cap_l = chi[j];
    lv.cap_r = chi[j + 1];
    const cplx<R>* Bj = B + st->site_off[j];
    const int tl = (lv.cap_l + kTile - 1) / kTile, tr = (lv.cap_r + kTile - 1) / kTile;
    if (st->tc && std::max(chi[j], chi[j + 1]) >= kTcMinChi) {
      // complex64 on the tensor cores: diagonal parents by scaling, stored
      // environments and children as batched tcgen05 complex GEMMs (below
      // kTcMinChi a 128-row tile is mostly padding and the CUDA-core
      // kernels are faster)
      if (!launch_env_tc<R>(st, h, L, j, chi, Lprev, Bj, M, Lcur)) {
        set_error("energy: tensor-core launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        return MPS_ECUDA;
      }
    } else {
      {
        KernelScope k(c, MPS_K_ENV_M);
        env_m_kernel<R><<<(unsigned)((size_t)L.n_parents * tl * tr), blk, 0, s>>>(
            Lprev, Bj, st->d_lam + st->lam_off[j], st->d_chi, lv, M);
      }
      if (L.n_children) {
        KernelScope k(c, MPS_K_ENV_CHILD);
        env_child_kernel<R><<<(unsigned)((size_t)L.n_children * tr * tr), blk, 0, s>>>(M, Bj, st->d_chi, lv, Lcur);
      }
    }
    if (L.n_leaves) {
      KernelScope k(c, MPS_K_ENV_LEAF);
      env_leaf_kernel<R><<<(L.n_leaves + 7) / 8, 256, 0, s>>>(M, Bj, st->d_chi, lv, st->d_vals);
    }
    if (L.n_traces) {
      KernelScope k(c, MPS_K_ENV_TRACE);
      env_trace_kernel<R><<<(L.n_traces + 7) / 8, 256, 0, s>>>(Lcur, st->d_chi, lv, st->d_vals);
    }
    if (L.n_children) std::swap(Lprev, Lcur);
  }
  {
    KernelScope k(c, MPS_K_REDUCE);
    energy_reduce_kernel<<<1, 1024, 0, s>>>(st->d_vals, h->d_coeffs, nt, 0.0, st->tc ? &st->d_rep->tc_error : nullptr,
                                            d_out ? d_out : st->d_energy);
  }
  MPSV_CUDA(cudaGetLastError());
  return MPS_OK;
}

mps_status ham_energy_async(mps_state* st, mps_ham* h, double* d_out) {
  if (h->n != st->n || h->ctx->device != st->ctx->device) {
    set_error("energy: Hamiltonian on %d qubits (device %d), state has %d (device %d)", h->n, h->ctx->device, st->n,
              st->ctx->device);
    return MPS_EINVAL;
  }
  if (st->broken) {
    set_error("energy: state is inconsistent after an earlier failure; reset it");
    return MPS_ESTATE;
  }
  return st->fp32 ? energy_levels<float>(st, h, d_out) : energy_levels<double>(st, h, d_out);
}

static void destroy_ham(mps_ham* h) {
  if (!h) return;
  mps_ctx* c = h->ctx;
  DeviceGuard guard(c->device);
  cudaStreamSynchronize(c->stream);
  for (void* p : {(void*)h->d_parent_src, (void*)h->d_child, (void*)h->d_leaf, (void*)h->d_trace,
                  (void*)h->d_coeffs, (void*)h->d_dense, (void*)h->d_diag})
    dev_free(c, p);
  delete h;
}

}  // namespace mpsv

using namespace mpsv;

namespace mpsv {

cudaError_t queue_flags(mps_state* st, StateFlags* f) {
  f->not_converged = 0;
  f->tc_error = 0;
  return cudaMemcpyAsync(f, &st->d_rep->not_converged, sizeof(StateFlags), cudaMemcpyDeviceToHost, st->ctx->stream);
}

mps_status flags_status(const StateFlags& f, bool gates) {
  if (f.tc_error) {
    set_error("energy: a tensor-core contraction ran out of its bounded wait");
    return MPS_ETIMEOUT;
  }
  if (gates && f.not_converged) {
    set_error("%d truncation SVDs reached the Jacobi sweep cap; their results were used as they stand",
              f.not_converged);
    return MPS_ENOTCONV;
  }
  return MPS_OK;
}

}  // namespace mpsv

extern "C" {

mps_status mps_hamiltonian_create(mps_ctx* ctx, int32_t n_qubits, size_t n_terms, const uint8_t* ops,
                                  const double* coeffs, mps_ham** out) {
  if (!ctx || !out || (n_terms && (!ops || !coeffs))) {
    set_error("mps_hamiltonian_create: NULL argument");
    return MPS_EINVAL;
  }
  *out = nullptr;
  if (n_qubits < 2 || n_terms > (size_t)INT32_MAX) {
    set_error("mps_hamiltonian_create: n_qubits = %d, n_terms = %zu", n_qubits, n_terms);
    return MPS_EINVAL;
  }
  auto* h = new mps_ham();
  h->ctx = ctx;
  h->n = n_qubits;
  h->n_terms = (long long)n_terms;
  std::vector<int> parent_src;
  std::vector<int2> child;
  std::vector<int4> leaf;
  std::vector<int2> trace;
  std::vector<int2> dense;
  std::vector<int> diag;
  mps_status rc = build_trie(h, ops, coeffs, parent_src, child, leaf, trace, dense, diag);
  if (rc != MPS_OK) {
    delete h;
    return rc;
  }
  DeviceGuard guard(ctx->device);
  auto up = [&](void** dst, const void* src, size_t bytes) {
    if (rc != MPS_OK) return;
    rc = dev_alloc(ctx, dst, std::max<size_t>(bytes, 16));
    if (rc == MPS_OK && bytes) {
      cudaError_t e = cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream);
      if (e != cudaSuccess) rc = cuda_fail(e, "mps_hamiltonian_create upload");
    }
  };
  up((void**)&h->d_parent_src, parent_src.data(), parent_src.size() * sizeof(int));
  up((void**)&h->d_child, child.data(), child.size() * sizeof(int2));
  up((void**)&h->d_leaf, leaf.data(), leaf.size() * sizeof(int4));
  up((void**)&h->d_trace, trace.data(), trace.size() * sizeof(int2));
  up((void**)&h->d_dense, dense.data(), dense.size() * sizeof(int2));
  up((void**)&h->d_diag, diag.data(), diag.size() * sizeof(int));
  up((void**)&h->d_coeffs, coeffs, n_terms * sizeof(double));
  if (rc == MPS_OK) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "mps_hamiltonian_create");
  }
  if (rc != MPS_OK) {
    destroy_ham(h);
    return rc;
  }
  *out = h;
  return MPS_OK;
}

mps_status mps_hamiltonian_info(const mps_ham* h, int64_t* n_terms, int64_t* n_nodes, int64_t* max_level_nodes) {
  if (!h) {
    set_error("mps_hamiltonian_info: NULL Hamiltonian");
    return MPS_EINVAL;
  }
  if (n_terms) *n_terms = h->n_terms;
  if (n_nodes) *n_nodes = h->n_nodes;
  if (max_level_nodes) *max_level_nodes = h->max_level_nodes;
  return MPS_OK;
}

void mps_ham_destroy(mps_ham* h) { destroy_ham(h); }

mps_status mps_energy_async(mps_state* st, const mps_ham* h, double* d_energy_out) {
  if (!st || !h || !d_energy_out) {
    set_error("mps_energy_async: NULL argument");
    return MPS_EINVAL;
  }
  DeviceGuard guard(st->ctx->device);
  return ham_energy_async(st, const_cast<mps_ham*>(h), d_energy_out);
}

mps_status mps_energy(mps_state* st, const mps_ham* h, double* energy_out, double* norm_out) {
  if (!st || !h || !energy_out) {
    set_error("mps_energy: NULL argument");
    return MPS_EINVAL;
  }
  DeviceGuard guard(st->ctx->device);
  mps_ham* hh = const_cast<mps_ham*>(h);
  mps_status rc = ham_energy_async(st, hh, nullptr);
  if (rc != MPS_OK) return rc;
  MPSV_CUDA(cudaMemcpyAsync(energy_out, st->d_energy, sizeof(double), cudaMemcpyDeviceToHost, st->ctx->stream));
  StateFlags flags;
  MPSV_CUDA(queue_flags(st, &flags));
  if (norm_out) {
    // sum of lam^2 on bond 1 (the first inner bond; bond 0 is the trivial edge)
    const int b = st->n > 1 ? 1 : 0;
    std::vector<int> chi(st->n + 1);
    MPSV_CUDA(cudaMemcpyAsync(chi.data(), st->d_chi, (st->n + 1) * sizeof(int), cudaMemcpyDeviceToHost,
                              st->ctx->stream));
    MPSV_CUDA(cudaStreamSynchronize(st->ctx->stream));
    std::vector<double> lam(chi[b]);
    MPSV_CUDA(cudaMemcpyAsync(lam.data(), st->d_lam + st->lam_off[b], chi[b] * sizeof(double),
                              cudaMemcpyDeviceToHost, st->ctx->stream));
    MPSV_CUDA(cudaStreamSynchronize(st->ctx->stream));
    double s = 0.0;
    for (double v : lam) s += v * v;
    *norm_out = s;
  }
  MPSV_CUDA(cudaStreamSynchronize(st->ctx->stream));
  return flags_status(flags, false);
}

mps_status mps_expectations(mps_state* st, const mps_ham* h, double* values_out) {
  if (!st || !h || (!values_out && h->n_terms)) {
    set_error("mps_expectations: NULL argument");
    return MPS_EINVAL;
  }
  DeviceGuard guard(st->ctx->device);
  mps_ham* hh = const_cast<mps_ham*>(h);
  mps_status rc = ham_energy_async(st, hh, nullptr);
  if (rc != MPS_OK) return rc;
  if (h->n_terms)
    MPSV_CUDA(cudaMemcpyAsync(values_out, st->d_vals, h->n_terms * sizeof(double), cudaMemcpyDeviceToHost,
                              st->ctx->stream));
  StateFlags flags;
  MPSV_CUDA(queue_flags(st, &flags));
  MPSV_CUDA(cudaStreamSynchronize(st->ctx->stream));
  return flags_status(flags, false);
}

mps_status vqe_eval(mps_ctx* ctx, const vqe_request* reqs, size_t n, double* energies_out,
                    mps_status* status_out) {
  if (!ctx || (n && (!reqs || !energies_out))) {
    set_error("vqe_eval: NULL argument");
    return MPS_EINVAL;
  }
  DeviceGuard guard(ctx->device);
  mps_status first_bad = MPS_OK;
  for (size_t i = 0; i < n; ++i) {
    const vqe_request& r = reqs[i];
    mps_status rc = MPS_OK;
    if (!r.state || !r.circuit || !r.ham || r.state->ctx != ctx) {
      set_error("vqe_eval: request %zu has a NULL handle or another context", i);
      rc = MPS_EINVAL;
    }
    if (rc == MPS_OK) rc = state_reset(r.state, r.init_bits);
    if (rc == MPS_OK) rc = mps_apply_circuit_async(r.state, r.circuit, r.theta, 0);
    if (rc == MPS_OK) rc = ham_energy_async(r.state, const_cast<mps_ham*>(r.ham), nullptr);
    if (rc == MPS_OK) {
      cudaError_t e = cudaMemcpyAsync(&energies_out[i], r.state->d_energy, sizeof(double), cudaMemcpyDeviceToHost,
                                      ctx->stream);
      StateFlags flags;
      if (e == cudaSuccess) e = queue_flags(r.state, &flags);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      rc = e != cudaSuccess ? cuda_fail(e, "vqe_eval") : flags_status(flags, true);
    }
    if (rc != MPS_OK) {
      if (!status_has_result(rc)) energies_out[i] = 0.0;
      if (first_bad == MPS_OK) first_bad = rc;
    }
    if (status_out) status_out[i] = rc;
  }
  return first_bad;
}

}  // extern "C"

namespace mpsv {

// Shared body of vqe_eval_batch (host theta and energies, synchronising) and
// vqe_eval_batch_async (device theta and energies).
static mps_status run_batch(const vqe_request* reqs, size_t n, double* energies_out, mps_status* status_out,
                            bool on_device) {
  if (n && (!reqs || !energies_out)) {
    set_error("vqe_eval_batch: NULL argument");
    return MPS_EINVAL;
  }
  std::vector<mps_status> rc(n, MPS_OK);
  for (size_t i = 0; i < n; ++i) {
    const vqe_request& r = reqs[i];
    if (!r.state || !r.circuit || !r.ham || (!r.theta && r.circuit->n_params)) {
      set_error("vqe_eval_batch: request %zu has a NULL handle", i);
      rc[i] = MPS_EINVAL;
      continue;
    }
    for (size_t j = 0; j < i; ++j)
      if (reqs[j].state == r.state) {
        set_error("vqe_eval_batch: requests %zu and %zu share a state", j, i);
        rc[i] = MPS_EINVAL;
      }
    if (rc[i] == MPS_OK && (r.circuit->n != r.state->n || r.ham->n != r.state->n ||
                            r.circuit->ctx->device != r.state->ctx->device)) {
      set_error("vqe_eval_batch: request %zu mixes sizes or devices", i);
      rc[i] = MPS_EINVAL;
    }
  }
  // Reset, bind and gates.  The requests are grouped by context (a
  // context's stream and bookkeeping belong to one host thread) and the
  // groups are fed by up to 16 host threads, each going round-robin over
  // its requests gate by gate, so the host's launch rate does not cap the
  // number of evaluations in flight.
  std::vector<std::vector<size_t>> groups;
  {
    std::vector<mps_ctx*> keys;
    for (size_t i = 0; i < n; ++i) {
      if (rc[i] != MPS_OK) continue;
      mps_ctx* c = reqs[i].state->ctx;
      size_t gi = 0;
      while (gi < keys.size() && keys[gi] != c) ++gi;
      if (gi == keys.size()) {
        keys.push_back(c);
        groups.emplace_back();
      }
      groups[gi].push_back(i);
    }
  }
  const size_t hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t n_threads = std::min<size_t>({groups.size(), std::max<size_t>(1, hw / 2), 16});
  std::vector<std::string> errs(n_threads);
  auto work = [&](size_t t) {
    std::vector<size_t> mine;
    for (size_t gi = t; gi < groups.size(); gi += n_threads)
      for (size_t i : groups[gi]) mine.push_back(i);
    for (size_t i : mine) {
      const vqe_request& r = reqs[i];
      DeviceGuard guard(r.state->ctx->device);
      rc[i] = state_reset(r.state, r.init_bits);
      if (rc[i] == MPS_OK) rc[i] = state_bind_circuit(r.state, r.circuit, r.theta, on_device ? 1 : 0);
    }
    int max_gates = 0;
    for (size_t i : mine)
      if (rc[i] == MPS_OK) max_gates = std::max(max_gates, reqs[i].circuit->n_gates);
    for (int g = 0; g < max_gates; ++g) {
      for (size_t i : mine) {
        const vqe_request& r = reqs[i];
        if (rc[i] != MPS_OK || g >= r.circuit->n_gates) continue;
        DeviceGuard guard(r.state->ctx->device);
        rc[i] = state_apply_device_gates(r.state, r.state->d_bound + g, &r.circuit->q[g], &r.circuit->arity[g], 1);
        if (rc[i] != MPS_OK) r.state->broken = true;
      }
    }
    for (size_t i : mine)
      if (rc[i] != MPS_OK && errs[t].empty()) errs[t] = last_error();
  };
  if (n_threads <= 1) {
    if (!groups.empty()) work(0);
  } else {
    std::vector<std::thread> pool;
    for (size_t t = 1; t < n_threads; ++t) pool.emplace_back(work, t);
    work(0);
    for (auto& th : pool) th.join();
    for (auto& e : errs)
      if (!e.empty()) {
        set_error("%s", e.c_str());
        break;
      }
  }
  // energies (each reads its bond dimensions once), then the results
  std::vector<StateFlags> flags(n);
  for (size_t i = 0; i < n; ++i) {
    if (rc[i] != MPS_OK) continue;
    const vqe_request& r = reqs[i];
    DeviceGuard guard(r.state->ctx->device);
    rc[i] = ham_energy_async(r.state, const_cast<mps_ham*>(r.ham), on_device ? energies_out + i : nullptr);
    if (rc[i] == MPS_OK && !on_device) {
      cudaError_t e = cudaMemcpyAsync(&energies_out[i], r.state->d_energy, sizeof(double), cudaMemcpyDeviceToHost,
                                      r.state->ctx->stream);
      if (e == cudaSuccess) e = queue_flags(r.state, &flags[i]);
      if (e != cudaSuccess) rc[i] = cuda_fail(e, "vqe_eval_batch");
    }
  }
  mps_status first_bad = MPS_OK;
  for (size_t i = 0; i < n; ++i) {
    if (rc[i] == MPS_OK && !on_device) {
      DeviceGuard guard(reqs[i].state->ctx->device);
      cudaError_t e = cudaStreamSynchronize(reqs[i].state->ctx->stream);
      rc[i] = e != cudaSuccess ? cuda_fail(e, "vqe_eval_batch") : flags_status(flags[i], true);
    }
    if (rc[i] != MPS_OK) {
      if (!on_device && !status_has_result(rc[i])) energies_out[i] = 0.0;
      if (first_bad == MPS_OK) first_bad = rc[i];
    }
    if (status_out) status_out[i] = rc[i];
  }
  return first_bad;
}

}  // namespace mpsv

extern "C" {

mps_status vqe_eval_batch(const vqe_request* reqs, size_t n, double* energies_out, mps_status* status_out) {
  return run_batch(reqs, n, energies_out, status_out, false);
}

mps_status vqe_eval_batch_async(const vqe_request* reqs, size_t n, double* d_energies_out, mps_status* status_out) {
  return run_batch(reqs, n, d_energies_out, status_out, true);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Linear observables over one string set: reduced density matrices
// ---------------------------------------------------------------------------

struct mps_obs {
  mps_ctx* ctx = nullptr;  // the string set's context (owns the arrays below)
  const mps_ham* strings = nullptr;
  long long n_rows = 0, nnz = 0;
  long long* d_row_ptr = nullptr;
  int* d_cols = nullptr;
  double2* d_w = nullptr;
};

static void destroy_obs(mps_obs* o) {
  if (!o) return;
  mps_ctx* c = o->ctx;
  DeviceGuard guard(c->device);
  cudaStreamSynchronize(c->stream);
  for (void* p : {(void*)o->d_row_ptr, (void*)o->d_cols, (void*)o->d_w}) dev_free(c, p);
  delete o;
}

extern "C" {

mps_status mps_observables_create(const mps_ham* strings, size_t n_rows, const int64_t* row_ptr,
                                  const int32_t* cols, const double* weights, mps_obs** out) {
  if (!strings || !out || !row_ptr) {
    set_error("mps_observables_create: NULL argument");
    return MPS_EINVAL;
  }
  *out = nullptr;
  if (n_rows > (size_t)INT32_MAX * 8) {
    set_error("mps_observables_create: n_rows = %zu is too large", n_rows);
    return MPS_EINVAL;
  }
  if (row_ptr[0] != 0) {
    set_error("mps_observables_create: row_ptr[0] = %lld, must be 0", (long long)row_ptr[0]);
    return MPS_EINVAL;
  }
  for (size_t r = 0; r < n_rows; ++r)
    if (row_ptr[r + 1] < row_ptr[r]) {
      set_error("mps_observables_create: row_ptr decreases at row %zu", r);
      return MPS_EINVAL;
    }
  const long long nnz = row_ptr[n_rows];
  if (nnz > 0 && (!cols || !weights)) {
    set_error("mps_observables_create: NULL cols or weights for %lld entries", nnz);
    return MPS_EINVAL;
  }
  for (long long e = 0; e < nnz; ++e) {
    if (cols[e] < 0 || cols[e] >= strings->n_terms) {
      set_error("mps_observables_create: cols[%lld] = %d is not a string index (0..%lld)", e, cols[e],
                strings->n_terms - 1);
      return MPS_EINVAL;
    }
    if (!std::isfinite(weights[2 * e]) || !std::isfinite(weights[2 * e + 1])) {
      set_error("mps_observables_create: weight %lld is not finite", e);
      return MPS_EINVAL;
    }
  }
  mps_ctx* c = strings->ctx;
  DeviceGuard guard(c->device);
  auto* o = new mps_obs();
  o->ctx = c;
  o->strings = strings;
  o->n_rows = (long long)n_rows;
  o->nnz = nnz;
  mps_status rc = dev_alloc(c, (void**)&o->d_row_ptr, (n_rows + 1) * sizeof(long long));
  if (rc == MPS_OK) rc = dev_alloc(c, (void**)&o->d_cols, (size_t)nnz * sizeof(int));
  if (rc == MPS_OK) rc = dev_alloc(c, (void**)&o->d_w, (size_t)nnz * sizeof(double2));
  if (rc == MPS_OK) {
    cudaError_t e = cudaMemcpy(o->d_row_ptr, row_ptr, (n_rows + 1) * sizeof(long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nnz)
      e = cudaMemcpy(o->d_cols, cols, (size_t)nnz * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nnz)
      e = cudaMemcpy(o->d_w, weights, (size_t)nnz * sizeof(double2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) rc = cuda_fail(e, "mps_observables_create: upload");
  }
  if (rc != MPS_OK) {
    destroy_obs(o);
    return rc;
  }
  *out = o;
  return MPS_OK;
}

mps_status mps_observables_eval(mps_state* st, const mps_obs* o, double* values_out) {
  if (!st || !o || (!values_out && o->n_rows)) {
    set_error("mps_observables_eval: NULL argument");
    return MPS_EINVAL;
  }
  if (o->ctx->device != st->ctx->device) {
    set_error("mps_observables_eval: observables on device %d, state on device %d", o->ctx->device,
              st->ctx->device);
    return MPS_EINVAL;
  }
  DeviceGuard guard(st->ctx->device);
  mps_status rc = ham_energy_async(st, const_cast<mps_ham*>(o->strings), nullptr);
  if (rc != MPS_OK) return rc;
  if ((size_t)o->n_rows > st->obs_cap || !st->d_obs) {
    MPSV_CUDA(cudaStreamSynchronize(st->ctx->stream));
    dev_free(st->ctx, st->d_obs);
    st->d_obs = nullptr;
    st->obs_cap = 0;
    rc = dev_alloc(st->ctx, (void**)&st->d_obs, std::max<size_t>(16, (size_t)o->n_rows * sizeof(double2)));
    if (rc != MPS_OK) return rc;
    st->obs_cap = (size_t)o->n_rows;
  }
  cudaStream_t s = st->ctx->stream;
  if (o->n_rows) {
    {
      KernelScope k(st->ctx, MPS_K_REDUCE);
      const long long blocks = (o->n_rows + 7) / 8;  // 8 warps (rows) per 256-thread block
      observables_kernel<<<(unsigned)blocks, 256, 0, s>>>(st->d_vals, o->d_row_ptr, o->d_cols, o->d_w, o->n_rows,
                                                           st->d_obs);
    }
    MPSV_CUDA(cudaGetLastError());
    MPSV_CUDA(cudaMemcpyAsync(values_out, st->d_obs, (size_t)o->n_rows * sizeof(double2), cudaMemcpyDeviceToHost,
                              s));
  }
  StateFlags flags;
  MPSV_CUDA(queue_flags(st, &flags));
  MPSV_CUDA(cudaStreamSynchronize(s));
  return flags_status(flags, false);
}

void mps_observables_destroy(mps_obs* o) { destroy_obs(o); }

}  // extern "C"
