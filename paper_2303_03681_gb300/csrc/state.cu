// Contexts, states, gates and circuit templates of libmpsvqe.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>

#include "gate_kernels.cuh"
#include "internal.h"
#include "svd_cluster.cuh"

namespace mpsv {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

const char* last_error() { return g_last_error.c_str(); }

mps_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? MPS_ENOMEM : MPS_ECUDA;
}

mps_status dev_alloc(mps_ctx* ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (ctx->alloc_limit && ctx->allocated + bytes > ctx->alloc_limit) {
    set_error("allocation of %zu bytes exceeds the context cap (%zu of %zu in use)", bytes, ctx->allocated,
              ctx->alloc_limit);
    return MPS_ENOMEM;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    set_error("cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    return MPS_ENOMEM;
  }
  ctx->allocated += bytes;
  ctx->allocs[*p] = bytes;
  return MPS_OK;
}

void dev_free(mps_ctx* ctx, void* p) {
  if (!p) return;
  auto it = ctx->allocs.find(p);
  if (it != ctx->allocs.end()) {
    ctx->allocated -= it->second;
    ctx->allocs.erase(it);
  }
  cudaFree(p);
}

KernelScope::KernelScope(mps_ctx* ctx, int k) : c(ctx), kind(k) {
  if (c->capturing) {
    // inside a graph capture: counted per replay, timed with the graph's own events
    c->capturing->counts[k] += 1;
    if (!(c->prof_mask & (1u << k))) return;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      cudaGetLastError();
      if (a) cudaEventDestroy(a);
      a = b = nullptr;
      return;
    }
    cudaEventRecordWithFlags(a, c->stream, cudaEventRecordExternal);  // an event-record node of the graph
    return;
  }
  c->launches[k] += 1;
  if (!(c->prof_mask & (1u << k))) return;
  for (cudaEvent_t* e : {&a, &b}) {
    if (!c->pool.empty()) {
      *e = c->pool.back();
      c->pool.pop_back();
    } else if (cudaEventCreate(e) != cudaSuccess) {
      cudaGetLastError();
      *e = nullptr;
    }
  }
  if (a && b) cudaEventRecord(a, c->stream);
}

KernelScope::~KernelScope() {
  if (c->capturing) {
    if (a && b) {
      cudaEventRecordWithFlags(b, c->stream, cudaEventRecordExternal);
      c->capturing->timing.push_back({kind, a, b});
    }
    return;
  }
  if (!a || !b) {
    if (a) c->pool.push_back(a);
    if (b) c->pool.push_back(b);
    return;
  }
  cudaEventRecord(b, c->stream);
  c->pending.push_back({kind, a, b});
}

static void collect_profile(mps_ctx* c) {
  for (auto& p : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->ms[p.kind] += ms;
      c->timed[p.kind] += 1;
    } else {
      cudaGetLastError();
    }
    c->pool.push_back(p.a);
    c->pool.push_back(p.b);
  }
  c->pending.clear();
  // graph replays: the events hold the last replay's times, taken for every
  // replay since the previous collection
  for (CircuitGraph* g : c->graph_watch) {
    if (g->unread <= 0) continue;
    for (auto& t : g->timing) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
        c->ms[t.kind] += (double)ms * g->unread;
        c->timed[t.kind] += g->unread;
      } else {
        cudaGetLastError();
      }
    }
    g->unread = 0;
  }
  c->graph_watch.clear();
}

void graph_destroy(mps_ctx* c, CircuitGraph* g) {
  if (!g) return;
  for (size_t i = 0; i < c->graph_watch.size(); ++i)
    if (c->graph_watch[i] == g) {
      c->graph_watch.erase(c->graph_watch.begin() + i);
      break;
    }
  for (auto& t : g->timing) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  if (g->exec) cudaGraphExecDestroy(g->exec);
  delete g;
}

static int bond_cap(int b, int n, int chi_max) {
  int e = std::min(b, n - b);
  if (e >= 30) return chi_max;
  return std::min(chi_max, 1 << e);
}

// ---------------------------------------------------------------------------
// kernel launch helpers
// ---------------------------------------------------------------------------
template <typename R> static cplx<R>* site_ptr(mps_state* st, int s) {
  return reinterpret_cast<cplx<R>*>(st->d_B) + st->site_off[s];
}

template <typename S> static size_t svd_smem_bytes(int mcap, int ncap, bool use_smem) {
  size_t b = (size_t)ncap * (sizeof(double) + sizeof(int)) + 64;
  if (use_smem) b += ((size_t)mcap * ncap + (size_t)ncap * ncap) * sizeof(cplx<S>);
  return b;
}

static size_t max_dyn_smem() {
  static size_t v = 0;
  static std::once_flag f;
  std::call_once(f, [] {
    int dev = 0, val = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&val, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    v = (size_t)val;
  });
  return v;
}

template <typename S, typename R> static void svd_set_attr() {
  static std::once_flag f;
  std::call_once(f, [] {
    cudaFuncSetAttribute(svd_truncate_kernel<S, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(max_dyn_smem() - 1024));
  });
}

// Launch plan of the cluster Jacobi SVD for a theta with up to mcap rows and
// ncap columns (A = C~, stacked columns [A; V] of length mcap + ncap), or
// P = 0 when the single-CTA kernel is used.  The stacked columns stay in
// shared memory when the capacities allow; otherwise they live in the
// state's global workspace, and the kernel still keeps them in shared
// memory whenever the actual bond dimensions fit the allocation given here.
struct SvdPlan {
  int P = 0;
  int threads = 0;
  size_t smem = 0;
  bool global = false;
};

template <typename S, typename R> static SvdPlan cluster_svd_plan(int mcap, int ncap) {
  SvdPlan pl;
  // FP64 runs at 2 FMA/clk/SM on this part, so even small FP64 thetas gain
  // from spreading their columns over several SMs; FP32 ones only from 96.
  if (ncap < (sizeof(S) == 8 ? 32 : 96)) return pl;
  static int max16 = -1;
  static std::once_flag f;
  std::call_once(f, [] {
    cudaFuncSetAttribute(svd_cluster_kernel<S, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(max_dyn_smem() - 1024));
    cudaFuncSetAttribute(svd_cluster_kernel<S, R>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(kClusterMaxThreads<S>);
    cfg.dynamicSmemBytes = max_dyn_smem() - 2048;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, svd_cluster_kernel<S, R>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      n = 0;
    }
    max16 = n;
  });
  const size_t lim = max_dyn_smem() - 2048;
  if constexpr (sizeof(S) == 4) {
    // FP32 pair steps are latency-bound: few CTAs (fewer rounds and cluster
    // barriers) with 16 warps each, so that concurrent evaluations find SMs
    // free.  Columns stay in shared memory whenever the actual sizes fit.
    const int P = 4, b = (ncap + 2 * P - 1) / (2 * P);
    pl.P = P;
    pl.threads = 512;
    ClusterSvdSmem<S> L(b, mcap + ncap, 2 * P * b, pl.threads);
    if (L.total <= lim) {
      pl.smem = L.total;
    } else {
      pl.global = true;
      pl.smem = std::min(lim, std::max(ClusterSvdSmem<S>(b, 0, 2 * P * b, pl.threads).total, (size_t)160 * 1024));
    }
    return pl;
  } else {
  // FP64 sweeps: at most 8 CTAs of up to 8 warps (one column pair each), so
  // that a block holds enough pairs to keep its SM's FP64 units busy; with
  // many evaluations in flight, 16 CTAs of 4 busy warps left most SMs waiting
  // at cluster barriers (0.47 against 0.70 evaluations/s at 32 streams)
  for (int P = ncap < 64 ? 4 : 8; P <= 8; P *= 2) {
    if (P == 16 && max16 <= 0) break;
    const int b = (ncap + 2 * P - 1) / (2 * P);
    ClusterSvdSmem<S> L(b, mcap + ncap, 2 * P * b, 32 * b);
    if (L.total <= lim && 32 * b <= 512) {
      pl.P = P;
      pl.threads = std::min(32 * b, kClusterMaxThreads<S>);
      pl.smem = L.total;
      return pl;
    }
  }
  // columns too long for shared memory at the capacity: a global workspace,
  // and the whole shared memory of the CTA so that the actual sizes use it
  // whenever they fit
  const int P = 8;
  const int b = (ncap + 2 * P - 1) / (2 * P);
  pl.P = P;
  pl.threads = std::min(32 * b, kClusterMaxThreads<S>);
  pl.global = true;
  pl.smem = lim;
  return pl;
  }
}

// The truncation SVD of one theta (bond capacities mcap x ncap): the
// cluster kernel when the plan has CTAs (it reads the row-major C and the
// lam_l row weights itself; gbuf is its global workspace), else the
// single-CTA kernel on the column-major lam-scaled copy A with the V
// workspace.  Writes B~_{q+1} = V^H rows, lam_{q+1}, chi[q+1] and the report.
template <typename R, typename S>
static void launch_svd(mps_ctx* ctx, const SvdPlan& plan, int mcap, int ncap, const SvdParams& p,
                       const cplx<R>* Cm, cplx<S>* A, cplx<S>* V, const double* lam_l, int* chi, int q,
                       cplx<R>* Bnext, double* lam_next, DevReport* rep, cudaStream_t s) {
  KernelScope k(ctx, MPS_K_SVD);
  if (plan.P) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(plan.P);
    cfg.blockDim = dim3(plan.threads);
    cfg.dynamicSmemBytes = plan.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = plan.P;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, svd_cluster_kernel<S, R>, Cm, lam_l, chi, q, p, Bnext, lam_next, rep,
                       plan.global ? A : (cplx<S>*)nullptr, (unsigned)plan.smem);
    return;
  }
  const size_t full = svd_smem_bytes<S>(mcap, ncap, true);
  const bool use_smem = full + 2048 <= max_dyn_smem();
  const size_t smem = svd_smem_bytes<S>(mcap, ncap, use_smem);
  svd_set_attr<S, R>();
  const int warps = std::min(32, std::max(1, ncap / 2));
  svd_truncate_kernel<S, R><<<1, 32 * warps, smem, s>>>(A, V, use_smem ? 1 : 0, chi, q, p, Bnext, lam_next, rep);
}

template <typename R, typename S>
static void launch_two_qubit(mps_state* st, const DevGate* g, int q, cudaStream_t s) {
  const int cap_l = st->cap[q], cap_m = st->cap[q + 1], cap_r = st->cap[q + 2];
  const dim3 blk(kTile, kTile);
  const dim3 g1((cap_r + kTile - 1) / kTile, (cap_l + kTile - 1) / kTile);
  const SvdPlan plan = cluster_svd_plan<S, R>(2 * cap_l, 2 * cap_r);
  const int P = plan.P;
  // split-product tensor-core contractions (complex64 states): the cluster
  // SVD reads C itself, so they serve the bonds where it runs
  const bool tcg = sizeof(R) == 4 && P && tc_gates_used(st, q);
  if (tcg) {
    tc_theta(st, g, q, s);
  } else {
    KernelScope k(st->ctx, MPS_K_THETA);
    theta_kernel<R, S><<<g1, blk, 0, s>>>(site_ptr<R>(st, q), site_ptr<R>(st, q + 1), g,
                                          st->d_lam + st->lam_off[q], st->d_chi, q,
                                          reinterpret_cast<cplx<R>*>(st->d_C),
                                          P ? nullptr : reinterpret_cast<cplx<S>*>(st->d_A));
  }
  SvdParams p;
  p.chi_max = st->cfg.chi_max;
  p.max_sweeps = st->cfg.svd_max_sweeps > 0 ? st->cfg.svd_max_sweeps : 60;
  p.trunc_rel = st->cfg.trunc_rel;
  p.tol = st->cfg.svd_tol;
  p.mixed = st->cfg.svd_fp64 == 2 ? 0 : 1;
  const dim3 g3((cap_m + kTile - 1) / kTile, (2 * cap_l + kTile - 1) / kTile);
  const cplx<R>* Cm = reinterpret_cast<const cplx<R>*>(st->d_C);
  launch_svd<R, S>(st->ctx, plan, 2 * cap_l, 2 * cap_r, p, Cm, reinterpret_cast<cplx<S>*>(st->d_A),
                   reinterpret_cast<cplx<S>*>(st->d_V), st->d_lam + st->lam_off[q], st->d_chi, q,
                   site_ptr<R>(st, q + 1), st->d_lam + st->lam_off[q + 1], st->d_rep, s);
  if (tcg) {
    tc_g3(st, q, s);
  } else {
    KernelScope k(st->ctx, MPS_K_G3);
    g3_kernel<R><<<g3, blk, 0, s>>>(reinterpret_cast<cplx<R>*>(st->d_C), site_ptr<R>(st, q + 1), st->d_chi, q,
                                    st->d_rep, site_ptr<R>(st, q));
  }
}

template <typename R>
static void launch_one_qubit(mps_state* st, const DevGate* g, int q, cudaStream_t s) {
  const int tot = st->cap[q] * st->cap[q + 1];
  KernelScope k(st->ctx, MPS_K_GATE1);
  gate1_kernel<R><<<(tot + 255) / 256, 256, 0, s>>>(site_ptr<R>(st, q), g, st->d_chi, q);
}

mps_status state_apply_device_gates(mps_state* st, const DevGate* d_gates, const int* q, const int* arity,
                                    size_t n) {
  cudaStream_t s = st->ctx->stream;
  for (size_t i = 0; i < n; ++i) {
    const DevGate* g = d_gates + i;
    if (arity[i] == 1) {
      if (st->fp32)
        launch_one_qubit<float>(st, g, q[i], s);
      else
        launch_one_qubit<double>(st, g, q[i], s);
    } else {
      if (st->fp32) {
        if (st->svd64)
          launch_two_qubit<float, double>(st, g, q[i], s);
        else
          launch_two_qubit<float, float>(st, g, q[i], s);
      } else {
        if (st->svd64)
          launch_two_qubit<double, double>(st, g, q[i], s);
        else
          launch_two_qubit<double, float>(st, g, q[i], s);
      }
    }
  }
  MPSV_CUDA(cudaGetLastError());
  return MPS_OK;
}

mps_status state_reset(mps_state* st, const uint8_t* bits) {
  cudaStream_t s = st->ctx->stream;
  std::vector<uint8_t> hb(st->n, 0);
  if (bits) {
    for (int i = 0; i < st->n; ++i) {
      if (bits[i] > 1) {
        set_error("init_bits[%d] = %d is not 0 or 1", i, (int)bits[i]);
        return MPS_EINVAL;
      }
      hb[i] = bits[i];
    }
  }
  if (hb != st->last_bits) {
    MPSV_CUDA(cudaMemcpyAsync(st->d_bits, hb.data(), st->n, cudaMemcpyHostToDevice, s));
    MPSV_CUDA(cudaStreamSynchronize(s));  // hb is a stack copy
    st->last_bits = hb;
  }
  const int threads = 256, blocks = (st->n + 1 + threads - 1) / threads;
  KernelScope k(st->ctx, MPS_K_SETUP);
  if (st->fp32)
    reset_kernel<float><<<blocks, threads, 0, s>>>(reinterpret_cast<float2*>(st->d_B), st->d_site_off, st->d_lam,
                                                   st->d_lam_off, st->d_chi, st->d_bits, st->n, st->d_rep);
  else
    reset_kernel<double><<<blocks, threads, 0, s>>>(reinterpret_cast<double2*>(st->d_B), st->d_site_off, st->d_lam,
                                                    st->d_lam_off, st->d_chi, st->d_bits, st->n, st->d_rep);
  MPSV_CUDA(cudaGetLastError());
  st->broken = false;
  st->nc_seen = 0;
  return MPS_OK;
}

// Workspace for the bound gates and theta, and theta copied in (stream-ordered).
static mps_status state_upload_theta(mps_state* st, const mps_circuit* c, const double* theta, int theta_on_device) {
  mps_ctx* ctx = st->ctx;
  cudaStream_t s = ctx->stream;
  if ((size_t)c->n_gates > st->bound_cap) {
    dev_free(ctx, st->d_bound);
    st->d_bound = nullptr;
    st->bound_cap = 0;
    mps_status rc = dev_alloc(ctx, (void**)&st->d_bound, std::max<size_t>(1, c->n_gates) * sizeof(DevGate));
    if (rc != MPS_OK) return rc;
    st->bound_cap = c->n_gates;
  }
  if ((size_t)c->n_params > st->theta_cap || !st->d_theta) {
    dev_free(ctx, st->d_theta);
    st->d_theta = nullptr;
    st->theta_cap = 0;
    mps_status rc = dev_alloc(ctx, (void**)&st->d_theta, std::max(1, c->n_params) * sizeof(double));
    if (rc != MPS_OK) return rc;
    st->theta_cap = std::max(1, c->n_params);
  }
  if (c->n_params)
    MPSV_CUDA(cudaMemcpyAsync(st->d_theta, theta, c->n_params * sizeof(double),
                              theta_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  return MPS_OK;
}

static void launch_bind(mps_state* st, const mps_circuit* c) {
  if (!c->n_gates) return;
  KernelScope k(st->ctx, MPS_K_SETUP);
  bind_kernel<<<c->n_gates, 32, 0, st->ctx->stream>>>(c->d_tmpl, c->n_gates, st->d_theta, st->d_bound);
}

mps_status state_bind_circuit(mps_state* st, const mps_circuit* c, const double* theta, int theta_on_device) {
  mps_status rc = state_upload_theta(st, c, theta, theta_on_device);
  if (rc != MPS_OK) return rc;
  launch_bind(st, c);
  MPSV_CUDA(cudaGetLastError());
  return MPS_OK;
}

// One-time launch attributes (shared-memory opt-ins, the 16-CTA cluster
// occupancy query) set before a capture, outside it.
template <typename R, typename S> static void prime_launch_attrs() {
  svd_set_attr<S, R>();
  (void)cluster_svd_plan<S, R>(256, 256);
}

static void prime_launch_attrs(const mps_state* st) {
  if (st->fp32)
    st->svd64 ? prime_launch_attrs<float, double>() : prime_launch_attrs<float, float>();
  else
    st->svd64 ? prime_launch_attrs<double, double>() : prime_launch_attrs<double, float>();
}

mps_status state_run_circuit(mps_state* st, const mps_circuit* c, const double* theta, int theta_on_device) {
  mps_ctx* ctx = st->ctx;
  cudaStream_t s = ctx->stream;
  mps_status rc = state_upload_theta(st, c, theta, theta_on_device);
  if (rc != MPS_OK || !c->n_gates) return rc;
  if (!ctx->use_graphs) {
    launch_bind(st, c);
    return state_apply_device_gates(st, st->d_bound, c->q.data(), c->arity.data(), c->n_gates);
  }
  CircuitGraph* g = st->graph;
  const bool hit = g && g->exec && g->circ_serial == c->serial && g->theta_ptr == st->d_theta &&
                   g->bound_ptr == st->d_bound && g->mask == ctx->prof_mask;
  if (!hit) {
    if (g) {
      MPSV_CUDA(cudaStreamSynchronize(s));
      collect_profile(ctx);
      graph_destroy(ctx, g);
      st->graph = nullptr;
    }
    g = new CircuitGraph();
    g->circ_serial = c->serial;
    g->theta_ptr = st->d_theta;
    g->bound_ptr = st->d_bound;
    g->mask = ctx->prof_mask;
    prime_launch_attrs(st);
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
      delete g;
      return cuda_fail(e, "cudaStreamBeginCapture");
    }
    ctx->capturing = g;
    launch_bind(st, c);
    rc = state_apply_device_gates(st, st->d_bound, c->q.data(), c->arity.data(), c->n_gates);
    ctx->capturing = nullptr;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(s, &graph);
    if (rc == MPS_OK && e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (rc != MPS_OK || e != cudaSuccess) {
      graph_destroy(ctx, g);
      return rc != MPS_OK ? rc : cuda_fail(e, "circuit graph capture");
    }
    st->graph = g;
  }
  MPSV_CUDA(cudaGraphLaunch(g->exec, s));
  g->unread += 1;
  for (int k = 0; k < MPS_K_COUNT; ++k) ctx->launches[k] += g->counts[k];
  bool watched = false;
  for (CircuitGraph* w : ctx->graph_watch) watched |= (w == g);
  if (!watched) ctx->graph_watch.push_back(g);
  return MPS_OK;
}

static void destroy_state(mps_state* st) {
  if (!st) return;
  mps_ctx* c = st->ctx;
  DeviceGuard guard(c->device);
  cudaStreamSynchronize(c->stream);
  if (st->graph) {
    collect_profile(c);
    graph_destroy(c, st->graph);
    st->graph = nullptr;
  }
  tc_gates_free(st);
  for (void* p : {st->d_B, (void*)st->d_lam, (void*)st->d_chi, (void*)st->d_site_off, (void*)st->d_lam_off,
                  (void*)st->d_bits, (void*)st->d_rep, st->d_C, st->d_A, st->d_V, (void*)st->d_gates,
                  (void*)st->d_bound, (void*)st->d_theta, st->d_L[0], st->d_L[1], st->d_M, (void*)st->d_vals,
                  (void*)st->d_energy, (void*)st->d_obs})
    dev_free(c, p);
  delete st;
}

static void host_gate_to_dev(const mps_gate& g, DevGate& d) {
  std::memset(&d, 0, sizeof(d));
  d.q = g.q;
  d.arity = g.arity;
  const int cnt = g.arity == 1 ? 4 : 16;
  for (int e = 0; e < cnt; ++e) d.u[e] = make_double2(g.u[2 * e], g.u[2 * e + 1]);
}

// ---- workspace and kernels of mps_truncated_svd (one theta on its own)
struct SvdWork {
  int mcap = 0, ncap = 0, sbytes = 0;
  int* d_chi = nullptr;
  DevReport* d_rep = nullptr;
  double* d_ones = nullptr;
  double* d_lam = nullptr;
  void* d_A = nullptr;
  void* d_V = nullptr;
};

void svd_work_free(mps_ctx* ctx) {
  SvdWork* w = ctx->svdw;
  if (!w) return;
  for (void* p : {(void*)w->d_chi, (void*)w->d_rep, (void*)w->d_ones, (void*)w->d_lam, w->d_A, w->d_V})
    dev_free(ctx, p);
  delete w;
  ctx->svdw = nullptr;
}

static __global__ void svd_setup_kernel(int* chi, int chi_l, int chi_r, DevReport* rep) {
  if (threadIdx.x != 0) return;
  chi[0] = chi_l;
  chi[1] = 0;
  chi[2] = chi_r;
  rep->discarded_weight = 0.0;
  rep->min_kept_sv = 1.0;
  rep->inv_norm = 1.0;
  rep->max_chi = 1;
  rep->degenerate_cuts = 0;
  rep->not_converged = 0;
  rep->tc_error = 0;
  rep->max_sweeps = 0;
  rep->two_qubit_gates = 0;
  rep->svd_flops = 0.0;
  rep->sweeps_fp32 = rep->sweeps_fp64 = 0;
  for (int i = 0; i < 4; ++i) rep->phase_cycles[i] = 0.0;
}

// column-major copy of the row-major theta (the single-CTA kernel's input; lam = 1)
template <typename R, typename S>
static __global__ void svd_c_to_a_kernel(const cplx<R>* __restrict__ C, int m, int n, cplx<S>* __restrict__ A) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)m * n) return;
  const int col = (int)(t / m), row = (int)(t % m);
  A[t] = ccast<cplx<S>>(C[(size_t)row * n + col]);
}

// the kept singular values without the renormalisation of the gate update
static __global__ void svd_finish_kernel(const int* chi, const DevReport* rep, const double* lam, double* s_out) {
  const int k = chi[1];
  const double nrm = 1.0 / rep->inv_norm;
  for (int a = threadIdx.x; a < k; a += blockDim.x) s_out[a] = lam[a] * nrm;
}

template <typename R, typename S>
static mps_status truncated_svd(mps_ctx* ctx, int m, int n, const void* C, const SvdParams& p, double* s_out,
                                void* Vh_out) {
  cudaStream_t s = ctx->stream;
  SvdWork* w = ctx->svdw;
  if (w && (m > w->mcap || n > w->ncap || (int)sizeof(S) > w->sbytes)) {
    MPSV_CUDA(cudaStreamSynchronize(s));
    svd_work_free(ctx);
    w = nullptr;
  }
  if (!w) {
    w = new SvdWork();
    ctx->svdw = w;
    w->mcap = m;
    w->ncap = n;
    w->sbytes = (int)sizeof(S);
    const size_t celem = sizeof(cplx<S>);
    mps_status rc = dev_alloc(ctx, (void**)&w->d_chi, 4 * sizeof(int));
    if (rc == MPS_OK) rc = dev_alloc(ctx, (void**)&w->d_rep, sizeof(DevReport));
    if (rc == MPS_OK) rc = dev_alloc(ctx, (void**)&w->d_ones, (size_t)m * sizeof(double));
    if (rc == MPS_OK) rc = dev_alloc(ctx, (void**)&w->d_lam, (size_t)n * sizeof(double));
    if (rc == MPS_OK)
      rc = dev_alloc(ctx, &w->d_A, std::max((size_t)m * n, cluster_svd_workspace(m, n, sizeof(S))) * celem);
    if (rc == MPS_OK) rc = dev_alloc(ctx, &w->d_V, (size_t)n * n * celem);
    if (rc == MPS_OK) {
      std::vector<double> ones(m, 1.0);
      cudaError_t e = cudaMemcpyAsync(w->d_ones, ones.data(), m * sizeof(double), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) rc = cuda_fail(e, "mps_truncated_svd set-up");
    }
    if (rc != MPS_OK) {
      svd_work_free(ctx);
      return rc;
    }
  }
  const SvdPlan plan = cluster_svd_plan<S, R>(m, n);
  const cplx<R>* Cm = static_cast<const cplx<R>*>(C);
  svd_setup_kernel<<<1, 32, 0, s>>>(w->d_chi, m / 2, n / 2, w->d_rep);
  if (!plan.P) {
    const size_t tot = (size_t)m * n;
    svd_c_to_a_kernel<R, S><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Cm, m, n, static_cast<cplx<S>*>(w->d_A));
  }
  launch_svd<R, S>(ctx, plan, m, n, p, Cm, static_cast<cplx<S>*>(w->d_A), static_cast<cplx<S>*>(w->d_V), w->d_ones,
                   w->d_chi, 0, static_cast<cplx<R>*>(Vh_out), w->d_lam, w->d_rep, s);
  svd_finish_kernel<<<1, 256, 0, s>>>(w->d_chi, w->d_rep, w->d_lam, s_out);
  MPSV_CUDA(cudaGetLastError());
  return MPS_OK;
}

}  // namespace mpsv

using namespace mpsv;

extern "C" {

const char* mps_last_error(void) { return mpsv::last_error(); }

const char* mps_version(void) { return "libmpsvqe 0.1.0 (sm_103a)"; }

mps_status mps_ctx_create(int device, void* cuda_stream, mps_ctx** out) {
  if (!out) {
    set_error("mps_ctx_create: out is NULL");
    return MPS_EINVAL;
  }
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    set_error("mps_ctx_create: no CUDA device %d (%d visible%s%s)", device, count, e != cudaSuccess ? ", " : "",
              e != cudaSuccess ? cudaGetErrorString(e) : "");
    return e != cudaSuccess ? MPS_ECUDA : MPS_EINVAL;
  }
  DeviceGuard guard(device);
  auto* c = new mps_ctx();
  c->device = device;
  if (cuda_stream) {
    c->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete c;
      return cuda_fail(e, "cudaStreamCreateWithFlags");
    }
    c->own_stream = true;
  }
  *out = c;
  return MPS_OK;
}

mps_status mps_ctx_synchronize(mps_ctx* ctx) {
  if (!ctx) {
    set_error("mps_ctx_synchronize: NULL context");
    return MPS_EINVAL;
  }
  DeviceGuard guard(ctx->device);
  MPSV_CUDA(cudaStreamSynchronize(ctx->stream));
  return MPS_OK;
}

mps_status mps_ctx_set_alloc_limit(mps_ctx* ctx, size_t bytes) {
  if (!ctx) {
    set_error("mps_ctx_set_alloc_limit: NULL context");
    return MPS_EINVAL;
  }
  ctx->alloc_limit = bytes;
  return MPS_OK;
}

mps_status mps_ctx_bytes_allocated(const mps_ctx* ctx, size_t* out) {
  if (!ctx || !out) {
    set_error("mps_ctx_bytes_allocated: NULL argument");
    return MPS_EINVAL;
  }
  *out = ctx->allocated;
  return MPS_OK;
}

mps_status mps_ctx_set_graphs(mps_ctx* ctx, int32_t enable) {
  if (!ctx) {
    set_error("mps_ctx_set_graphs: NULL context");
    return MPS_EINVAL;
  }
  ctx->use_graphs = enable != 0;
  return MPS_OK;
}

mps_status mps_ctx_profile(mps_ctx* ctx, uint32_t mask) {
  if (!ctx) {
    set_error("mps_ctx_profile: NULL context");
    return MPS_EINVAL;
  }
  ctx->prof_mask = mask;
  return MPS_OK;
}

mps_status mps_ctx_profile_read(mps_ctx* ctx, int32_t kind, int64_t* launches, int64_t* timed_launches, double* ms,
                                int32_t reset) {
  if (!ctx || kind < 0 || kind >= MPS_K_COUNT) {
    set_error("mps_ctx_profile_read: NULL context or kind %d outside 0..%d", kind, MPS_K_COUNT - 1);
    return MPS_EINVAL;
  }
  DeviceGuard guard(ctx->device);
  MPSV_CUDA(cudaStreamSynchronize(ctx->stream));
  collect_profile(ctx);
  if (launches) *launches = ctx->launches[kind];
  if (timed_launches) *timed_launches = ctx->timed[kind];
  if (ms) *ms = ctx->ms[kind];
  if (reset) {
    ctx->launches[kind] = 0;
    ctx->timed[kind] = 0;
    ctx->ms[kind] = 0.0;
  }
  return MPS_OK;
}

void mps_ctx_destroy(mps_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard guard(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  collect_profile(ctx);
  contract_work_free(ctx);
  svd_work_free(ctx);
  for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
  for (auto& kv : ctx->allocs) cudaFree(kv.first);
  ctx->allocs.clear();
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

mps_status mps_create(mps_ctx* ctx, int32_t n_qubits, const uint8_t* init_bits, const mps_config* cfg,
                      mps_state** out) {
  if (!ctx || !cfg || !out) {
    set_error("mps_create: NULL argument");
    return MPS_EINVAL;
  }
  *out = nullptr;
  if (n_qubits < 2 || n_qubits > 100000) {
    set_error("mps_create: n_qubits = %d outside [2, 100000]", n_qubits);
    return MPS_EINVAL;
  }
  if (cfg->chi_max < 1 || cfg->chi_max > 1024) {
    set_error("mps_create: chi_max = %d outside [1, 1024]", cfg->chi_max);
    return MPS_EINVAL;
  }
  if (cfg->precision < MPS_PREC_FP64 || cfg->precision > MPS_PREC_AUTO) {
    set_error("mps_create: unknown precision %d", cfg->precision);
    return MPS_EINVAL;
  }
  if (cfg->svd_fp64 < 0 || cfg->svd_fp64 > 2) {
    set_error("mps_create: svd_fp64 = %d is not 0, 1 or 2", cfg->svd_fp64);
    return MPS_EINVAL;
  }
  if (!(cfg->trunc_rel >= 0.0 && cfg->trunc_rel < 1.0)) {
    set_error("mps_create: trunc_rel = %g outside [0, 1)", cfg->trunc_rel);
    return MPS_EINVAL;
  }
  DeviceGuard guard(ctx->device);
  auto* st = new mps_state();
  st->ctx = ctx;
  st->n = n_qubits;
  st->cfg = *cfg;
  st->fp32 = cfg->precision != MPS_PREC_FP64;
  st->tc_gates = (cfg->precision == MPS_PREC_BF16X3 || cfg->precision == MPS_PREC_TF32X3 ||
                  cfg->precision == MPS_PREC_AUTO)
                     ? cfg->precision
                     : 0;
  st->svd64 = cfg->svd_fp64 != 0;
  st->tc = st->fp32 && (cfg->tensor_cores != 0 || st->tc_gates != 0);
  const int n = n_qubits;
  st->cap.resize(n + 1);
  for (int b = 0; b <= n; ++b) st->cap[b] = bond_cap(b, n, cfg->chi_max);
  st->site_off.resize(n);
  st->lam_off.resize(n + 1);
  size_t off = 0, loff = 0;
  size_t max_mn = 1, max_nn = 1, max_stack = 1;
  for (int s = 0; s < n; ++s) {
    st->site_off[s] = off;
    off += (size_t)st->cap[s] * 2 * st->cap[s + 1];
  }
  for (int b = 0; b <= n; ++b) {
    st->lam_off[b] = loff;
    loff += st->cap[b];
  }
  for (int q = 0; q + 1 < n; ++q) {
    const size_t m = 2 * (size_t)st->cap[q], nn = 2 * (size_t)st->cap[q + 2];
    max_mn = std::max(max_mn, m * nn);
    max_stack = std::max(max_stack, cluster_svd_workspace(m, nn, st->svd64 ? 8 : 4));
    max_nn = std::max(max_nn, nn * nn);
  }
  st->total_elems = off;
  st->total_lam = loff;
  const size_t celem = st->fp32 ? sizeof(float2) : sizeof(double2);
  const size_t selem = st->svd64 ? sizeof(double2) : sizeof(float2);
  mps_status rc = MPS_OK;
  auto A = [&](void** p, size_t bytes) {
    if (rc == MPS_OK) rc = dev_alloc(ctx, p, bytes);
  };
  A(&st->d_B, off * celem);
  A((void**)&st->d_lam, loff * sizeof(double));
  A((void**)&st->d_chi, (n + 1) * sizeof(int));
  A((void**)&st->d_site_off, n * sizeof(size_t));
  A((void**)&st->d_lam_off, (n + 1) * sizeof(size_t));
  A((void**)&st->d_bits, n);
  A((void**)&st->d_rep, sizeof(DevReport));
  A(&st->d_C, max_mn * celem);
  A(&st->d_A, std::max(max_mn, max_stack) * selem);  // theta copy, or the cluster SVD's stacked columns
  A(&st->d_V, max_nn * selem);
  if (rc == MPS_OK && st->tc_gates) rc = tc_gates_setup(st);
  if (rc != MPS_OK) {
    destroy_state(st);
    return rc;
  }
  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(st->d_site_off, st->site_off.data(), n * sizeof(size_t),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(st->d_lam_off, st->lam_off.data(), (n + 1) * sizeof(size_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(st->d_B, 0, off * celem, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(st->d_lam, 0, loff * sizeof(double), s);
  if (e != cudaSuccess) {
    destroy_state(st);
    return cuda_fail(e, "mps_create upload");
  }
  rc = state_reset(st, init_bits);
  if (rc != MPS_OK) {
    destroy_state(st);
    return rc;
  }
  *out = st;
  return MPS_OK;
}

mps_status mps_reset(mps_state* st, const uint8_t* init_bits) {
  if (!st) {
    set_error("mps_reset: NULL state");
    return MPS_EINVAL;
  }
  DeviceGuard guard(st->ctx->device);
  return state_reset(st, init_bits);
}

void mps_destroy(mps_state* st) { destroy_state(st); }

mps_status mps_get_report(mps_state* st, mps_report* out) {
  if (!st || !out) {
    set_error("mps_get_report: NULL argument");
    return MPS_EINVAL;
  }
  DeviceGuard guard(st->ctx->device);
  DevReport r;
  MPSV_CUDA(cudaMemcpyAsync(&r, st->d_rep, sizeof(r), cudaMemcpyDeviceToHost, st->ctx->stream));
  MPSV_CUDA(cudaStreamSynchronize(st->ctx->stream));
  out->discarded_weight = r.discarded_weight;
  out->min_kept_sv = r.min_kept_sv;
  out->max_chi = r.max_chi;
  out->degenerate_cuts = r.degenerate_cuts;
  out->svd_not_converged = r.not_converged;
  out->max_sweeps_used = r.max_sweeps;
  out->two_qubit_gates = r.two_qubit_gates;
  out->svd_flops = r.svd_flops;
  out->svd_sweeps_fp32 = r.sweeps_fp32;
  out->svd_sweeps_fp64 = r.sweeps_fp64;
  for (int i = 0; i < 4; ++i) out->svd_phase_cycles[i] = r.phase_cycles[i];
  return MPS_OK;
}

mps_status mps_apply_gates(mps_state* st, const mps_gate* gates, size_t n, mps_report* report) {
  if (!st || (!gates && n)) {
    set_error("mps_apply_gates: NULL argument");
    return MPS_EINVAL;
  }
  if (st->broken) {
    set_error("mps_apply_gates: state is inconsistent after an earlier failure; reset it");
    return MPS_ESTATE;
  }
  std::vector<int> q(n), ar(n);
  std::vector<DevGate> hg(n);
  for (size_t i = 0; i < n; ++i) {
    const mps_gate& g = gates[i];
    if (g.arity != 1 && g.arity != 2) {
      set_error("mps_apply_gates: gate %zu has arity %d", i, g.arity);
      return MPS_EINVAL;
    }
    if (g.q < 0 || g.q + g.arity > st->n) {
      set_error("mps_apply_gates: gate %zu on site %d (arity %d) outside 0..%d", i, g.q, g.arity, st->n - 1);
      return MPS_EINVAL;
    }
    q[i] = g.q;
    ar[i] = g.arity;
    host_gate_to_dev(g, hg[i]);
  }
  DeviceGuard guard(st->ctx->device);
  if (n > st->gates_cap) {
    dev_free(st->ctx, st->d_gates);
    st->d_gates = nullptr;
    st->gates_cap = 0;
    mps_status rc = dev_alloc(st->ctx, (void**)&st->d_gates, n * sizeof(DevGate));
    if (rc != MPS_OK) return rc;
    st->gates_cap = n;
  }
  if (n) {
    MPSV_CUDA(cudaMemcpyAsync(st->d_gates, hg.data(), n * sizeof(DevGate), cudaMemcpyHostToDevice,
                              st->ctx->stream));
    mps_status rc = state_apply_device_gates(st, st->d_gates, q.data(), ar.data(), n);
    if (rc != MPS_OK) {
      st->broken = true;
      return rc;
    }
  }
  cudaError_t e = cudaStreamSynchronize(st->ctx->stream);
  if (e != cudaSuccess) {
    st->broken = true;
    return cuda_fail(e, "mps_apply_gates");
  }
  mps_report r;
  mps_status rc = mps_get_report(st, &r);
  if (rc != MPS_OK) return rc;
  if (report) *report = r;
  // SVDs that reached the sweep cap since the host last looked (reset clears the count)
  const int fresh = r.svd_not_converged - st->nc_seen;
  st->nc_seen = r.svd_not_converged;
  if (fresh > 0) {
    set_error("mps_apply_gates: %d truncation SVDs reached the Jacobi sweep cap; their results were used as they stand",
              fresh);
    return MPS_ENOTCONV;
  }
  return MPS_OK;
}

mps_status mps_bond_dims(mps_state* st, int32_t* chi_out) {
  if (!st || !chi_out) {
    set_error("mps_bond_dims: NULL argument");
    return MPS_EINVAL;
  }
  DeviceGuard guard(st->ctx->device);
  MPSV_CUDA(cudaMemcpyAsync(chi_out, st->d_chi, (st->n + 1) * sizeof(int), cudaMemcpyDeviceToHost,
                            st->ctx->stream));
  MPSV_CUDA(cudaStreamSynchronize(st->ctx->stream));
  return MPS_OK;
}

mps_status mps_export(mps_state* st, double* tensors_out, size_t tensors_cap_doubles, double* lam_out,
                      size_t lam_cap) {
  if (!st || !tensors_out || !lam_out) {
    set_error("mps_export: NULL argument");
    return MPS_EINVAL;
  }
  DeviceGuard guard(st->ctx->device);
  std::vector<int> chi(st->n + 1);
  mps_status rc = mps_bond_dims(st, chi.data());
  if (rc != MPS_OK) return rc;
  size_t need = 0, need_lam = 0;
  for (int s = 0; s < st->n; ++s) need += 2 * (size_t)chi[s] * 2 * chi[s + 1];
  for (int b = 0; b <= st->n; ++b) need_lam += chi[b];
  if (need > tensors_cap_doubles || need_lam > lam_cap) {
    set_error("mps_export: buffers too small (need %zu tensor doubles, %zu lam doubles)", need, need_lam);
    return MPS_EINVAL;
  }
  const size_t celem = st->fp32 ? sizeof(float2) : sizeof(double2);
  std::vector<unsigned char> raw(st->total_elems * celem);
  std::vector<double> lam(st->total_lam);
  MPSV_CUDA(cudaMemcpyAsync(raw.data(), st->d_B, raw.size(), cudaMemcpyDeviceToHost, st->ctx->stream));
  MPSV_CUDA(cudaMemcpyAsync(lam.data(), st->d_lam, lam.size() * sizeof(double), cudaMemcpyDeviceToHost,
                            st->ctx->stream));
  MPSV_CUDA(cudaStreamSynchronize(st->ctx->stream));
  size_t o = 0;
  for (int s = 0; s < st->n; ++s) {
    const size_t cnt = (size_t)chi[s] * 2 * chi[s + 1];
    for (size_t e = 0; e < cnt; ++e) {
      if (st->fp32) {
        const float2 z = reinterpret_cast<const float2*>(raw.data())[st->site_off[s] + e];
        tensors_out[o++] = z.x;
        tensors_out[o++] = z.y;
      } else {
        const double2 z = reinterpret_cast<const double2*>(raw.data())[st->site_off[s] + e];
        tensors_out[o++] = z.x;
        tensors_out[o++] = z.y;
      }
    }
  }
  o = 0;
  for (int b = 0; b <= st->n; ++b)
    for (int a = 0; a < chi[b]; ++a) lam_out[o++] = lam[st->lam_off[b] + a];
  return MPS_OK;
}

// ---------------------------------------------------------------------------
// circuit templates
// ---------------------------------------------------------------------------
mps_status mps_circuit_create(mps_ctx* ctx, int32_t n_qubits, const mps_template_gate* gates, size_t n_gates,
                              int32_t n_params, mps_circuit** out) {
  if (!ctx || !out || (!gates && n_gates)) {
    set_error("mps_circuit_create: NULL argument");
    return MPS_EINVAL;
  }
  *out = nullptr;
  if (n_params < 0 || n_qubits < 2) {
    set_error("mps_circuit_create: n_qubits = %d, n_params = %d", n_qubits, n_params);
    return MPS_EINVAL;
  }
  std::vector<DevTmplGate> ht(n_gates);
  static std::atomic<uint64_t> next_serial{1};
  auto* c = new mps_circuit();
  c->serial = next_serial++;
  c->ctx = ctx;
  c->n = n_qubits;
  c->n_params = n_params;
  c->n_gates = (int)n_gates;
  c->q.resize(n_gates);
  c->arity.resize(n_gates);
  for (size_t i = 0; i < n_gates; ++i) {
    const mps_template_gate& g = gates[i];
    if ((g.arity != 1 && g.arity != 2) || g.q < 0 || g.q + g.arity > n_qubits || g.param >= n_params) {
      set_error("mps_circuit_create: gate %zu invalid (q=%d arity=%d param=%d)", i, g.q, g.arity, g.param);
      delete c;
      return MPS_EINVAL;
    }
    DevTmplGate& d = ht[i];
    std::memset(&d, 0, sizeof(d));
    d.q = g.q;
    d.arity = g.arity;
    d.param = g.param < 0 ? -1 : g.param;
    d.coeff = g.coeff;
    const int cnt = g.arity == 1 ? 4 : 16;
    for (int e = 0; e < cnt; ++e) {
      d.mp[e] = make_double2(g.m_plus[2 * e], g.m_plus[2 * e + 1]);
      d.mm[e] = make_double2(g.m_minus[2 * e], g.m_minus[2 * e + 1]);
    }
    c->q[i] = g.q;
    c->arity[i] = g.arity;
  }
  DeviceGuard guard(ctx->device);
  mps_status rc = dev_alloc(ctx, (void**)&c->d_tmpl, std::max<size_t>(1, n_gates) * sizeof(DevTmplGate));
  if (rc == MPS_OK && n_gates) {
    cudaError_t e = cudaMemcpyAsync(c->d_tmpl, ht.data(), n_gates * sizeof(DevTmplGate), cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "mps_circuit_create upload");
  }
  if (rc != MPS_OK) {
    dev_free(ctx, c->d_tmpl);
    delete c;
    return rc;
  }
  *out = c;
  return MPS_OK;
}

void mps_circuit_destroy(mps_circuit* c) {
  if (!c) return;
  DeviceGuard guard(c->ctx->device);
  cudaStreamSynchronize(c->ctx->stream);
  dev_free(c->ctx, c->d_tmpl);
  delete c;
}

mps_status mps_truncated_svd(mps_ctx* ctx, int32_t precision, int32_t m, int32_t n, const void* C, int32_t chi_max,
                             double trunc_rel, int32_t svd_fp64, double* s_out, void* Vh_out, int32_t* k_out,
                             mps_report* report) {
  if (!ctx || !C || !s_out || !Vh_out || !k_out) {
    set_error("mps_truncated_svd: NULL argument");
    return MPS_EINVAL;
  }
  if (precision != MPS_PREC_FP64 && precision != MPS_PREC_FP32) {
    set_error("mps_truncated_svd: precision %d is not MPS_PREC_FP64 or MPS_PREC_FP32", precision);
    return MPS_EINVAL;
  }
  if (m < 2 || n < 2 || m > 4096 || n > 4096 || (m & 1) || (n & 1)) {
    set_error("mps_truncated_svd: %d x %d theta: both sizes must be even and in 2..4096", m, n);
    return MPS_EINVAL;
  }
  if (chi_max < 1 || !(trunc_rel >= 0.0 && trunc_rel < 1.0) || svd_fp64 < 0 || svd_fp64 > 2) {
    set_error("mps_truncated_svd: chi_max = %d, trunc_rel = %g, svd_fp64 = %d", chi_max, trunc_rel, svd_fp64);
    return MPS_EINVAL;
  }
  DeviceGuard guard(ctx->device);
  SvdParams p;
  p.chi_max = chi_max;
  p.max_sweeps = 60;
  p.trunc_rel = trunc_rel;
  p.tol = 0.0;
  p.mixed = svd_fp64 == 2 ? 0 : 1;
  mps_status rc;
  if (precision == MPS_PREC_FP64)
    rc = svd_fp64 ? truncated_svd<double, double>(ctx, m, n, C, p, s_out, Vh_out)
                  : truncated_svd<double, float>(ctx, m, n, C, p, s_out, Vh_out);
  else
    rc = svd_fp64 ? truncated_svd<float, double>(ctx, m, n, C, p, s_out, Vh_out)
                  : truncated_svd<float, float>(ctx, m, n, C, p, s_out, Vh_out);
  if (rc != MPS_OK) return rc;
  DevReport r;
  int k = 0;
  MPSV_CUDA(cudaMemcpyAsync(&r, ctx->svdw->d_rep, sizeof(r), cudaMemcpyDeviceToHost, ctx->stream));
  MPSV_CUDA(cudaMemcpyAsync(&k, ctx->svdw->d_chi + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  MPSV_CUDA(cudaStreamSynchronize(ctx->stream));
  *k_out = k;
  if (report) {
    report->discarded_weight = r.discarded_weight;
    report->min_kept_sv = r.min_kept_sv;
    report->max_chi = r.max_chi;
    report->degenerate_cuts = r.degenerate_cuts;
    report->svd_not_converged = r.not_converged;
    report->max_sweeps_used = r.max_sweeps;
    report->two_qubit_gates = r.two_qubit_gates;
    report->svd_flops = r.svd_flops;
    report->svd_sweeps_fp32 = r.sweeps_fp32;
    report->svd_sweeps_fp64 = r.sweeps_fp64;
    for (int i = 0; i < 4; ++i) report->svd_phase_cycles[i] = r.phase_cycles[i];
  }
  if (r.not_converged) {
    set_error("mps_truncated_svd: the Jacobi SVD reached its sweep cap; the result is used as it stands");
    return MPS_ENOTCONV;
  }
  return MPS_OK;
}

mps_status mps_apply_circuit_async(mps_state* st, const mps_circuit* c, const double* theta, int theta_on_device) {
  if (!st || !c || (!theta && c->n_params)) {
    set_error("mps_apply_circuit_async: NULL argument");
    return MPS_EINVAL;
  }
  if (c->n != st->n || c->ctx->device != st->ctx->device) {
    set_error("mps_apply_circuit_async: circuit for %d qubits on device %d, state has %d on device %d", c->n,
              c->ctx->device, st->n, st->ctx->device);
    return MPS_EINVAL;
  }
  if (st->broken) {
    set_error("mps_apply_circuit_async: state is inconsistent after an earlier failure; reset it");
    return MPS_ESTATE;
  }
  DeviceGuard guard(st->ctx->device);
  mps_status rc = state_run_circuit(st, c, theta, theta_on_device);
  if (rc != MPS_OK) st->broken = true;
  return rc;
}

}  // extern "C"
