// Serving: continuous batching of VQE energy evaluations on one device.
//
// A native worker thread owns max_slots evaluation slots (a context with its
// own stream, a state and a pinned result word each).  Requests queue on the
// host; the worker admits them into free slots under the HBM budget, then in
// every pass issues a small group of gates for each admitted evaluation,
// starts the energy of evaluations whose gates have drained (the energy reads
// the bond dimensions, so it only starts once the stream is idle and never
// blocks the worker) and completes evaluations whose energy has arrived.  New
// requests join between gate groups while the others keep running.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

enum Phase { kQueued, kGates, kWaitGates, kWaitEnergy, kDone };

struct Request {
  uint64_t ticket = 0;
  int frag = 0;
  std::vector<double> theta;
  Clock::time_point t_submit;
  Phase phase = kQueued;
  int next_gate = 0;
  int slot = -1;
  double energy = 0.0;
  double latency_ms = 0.0;
  mps_status status = MPS_OK;
  std::string error;
};

struct Fragment {
  const mps_circuit* circ = nullptr;
  const mps_ham* ham = nullptr;
  std::vector<uint8_t> bits;
  mps_config cfg{};
  size_t est_bytes = 0;  // device bytes of one evaluation (estimate, then measured)
};

struct Slot {
  mps_ctx* ctx = nullptr;
  mps_state* st = nullptr;
  int frag = -1;
  Request* req = nullptr;
  double* h_energy = nullptr;  // pinned: [0] the energy, [1] the state's StateFlags
  cudaEvent_t chunk_ev[2] = {nullptr, nullptr};
  int chunks_in_flight = 0;
  int chunk_head = 0;
};

constexpr int kGatesPerTurn = 16;
constexpr size_t kMaxQueue = 1 << 16;

}  // namespace

struct mps_server {
  int device = 0;
  int max_slots = 1;
  size_t budget = 0;
  std::vector<Fragment> frags;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> live;
  uint64_t next_ticket = 1;
  std::thread worker;
  bool stop = false;
  long long completed = 0;
  int active = 0;
  size_t peak_bytes = 0;
};

namespace mpsv {
namespace {

size_t slots_bytes(const mps_server* s) {
  size_t b = 0;
  for (const Slot& sl : s->slots) b += sl.ctx ? sl.ctx->allocated : 0;
  return b;
}

// Upper bound of one evaluation's device memory for a fragment, from the bond
// capacities (the state arena, gate scratch, bound gates and the energy
// workspace at full capacity on every level).
size_t estimate_bytes(const Fragment& f) {
  const int n = f.ham->n;
  const int chi = f.cfg.chi_max;
  const size_t elem = f.cfg.precision == MPS_PREC_FP64 ? 16 : 8;
  auto cap = [&](int b) {
    const int e = std::min(b, n - b);
    return e >= 30 ? chi : std::min(chi, 1 << e);
  };
  size_t sites = 0, mn = 1;
  for (int s = 0; s < n; ++s) sites += (size_t)cap(s) * 2 * cap(s + 1);
  for (int q = 0; q + 1 < n; ++q) mn = std::max(mn, (size_t)4 * cap(q) * cap(q + 2));
  size_t env = 0;
  for (int j = 0; j < n; ++j) {
    const LevelHost& L = f.ham->levels[j];
    const size_t cl = cap(j), cr = cap(j + 1);
    env = std::max(env, 2 * (size_t)L.n_children * cr * cr * elem + (size_t)L.n_parents * 2 * cl * cr * elem);
  }
  // the operand planes of the split-product tensor-core contractions: A and B
  // pieces of (2 and 4) x maxcap rows by 4 maxcap FP32 values, hi and lo
  size_t tc = 0;
  if (f.cfg.precision != MPS_PREC_FP64 && f.cfg.precision != MPS_PREC_FP32) {
    int maxcap = 1;
    for (int b = 0; b <= n; ++b) maxcap = std::max(maxcap, cap(b));
    tc = 2 * (size_t)6 * (maxcap + 64) * (4 * (size_t)maxcap + 64) * 4;
  }
  return sites * elem + 3 * mn * 16 + (size_t)f.circ->n_gates * sizeof(DevGate) + env +
         (size_t)f.ham->n_terms * sizeof(double) + tc + (1 << 20);
}

void fail(mps_server* s, Slot& sl, mps_status rc) {
  std::lock_guard<std::mutex> lk(s->mu);
  Request* r = sl.req;
  r->status = rc;
  r->error = last_error();
  r->phase = kDone;
  r->latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - r->t_submit).count();
  sl.req = nullptr;
  s->active -= 1;
  s->completed += 1;
  if (sl.st) sl.st->broken = true;
  s->cv_done.notify_all();
}

// Puts a newly admitted request on its slot: a state of the fragment's shape
// (reused when the slot already holds one), reset, theta bound.
mps_status start(mps_server* s, Slot& sl) {
  Request* r = sl.req;
  const Fragment& f = s->frags[r->frag];
  if (sl.st && (sl.frag != r->frag || sl.st->broken)) {
    mps_destroy(sl.st);
    sl.st = nullptr;
  }
  if (!sl.st) {
    mps_status rc = mps_create(sl.ctx, f.ham->n, f.bits.data(), &f.cfg, &sl.st);
    if (rc != MPS_OK) return rc;
    sl.frag = r->frag;
  }
  mps_status rc = state_reset(sl.st, f.bits.data());
  if (rc == MPS_OK) rc = state_bind_circuit(sl.st, f.circ, r->theta.data(), 0);
  r->next_gate = 0;
  r->phase = kGates;
  sl.chunks_in_flight = 0;
  return rc;
}

void worker_loop(mps_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    // ---- admission (under the lock)
    std::vector<int> admitted;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop && s->active == 0 && s->queue.empty()) return;
      if (s->active == 0 && s->queue.empty()) {
        s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
        continue;
      }
      size_t held = slots_bytes(s);
      for (int i = 0; i < (int)s->slots.size() && !s->queue.empty(); ++i) {
        Slot& sl = s->slots[i];
        if (sl.req) continue;
        Request* r = s->queue.front();
        const Fragment& f = s->frags[r->frag];
        const size_t reuse = (sl.st && sl.frag == r->frag) ? sl.ctx->allocated : 0;
        const size_t need = f.est_bytes > reuse ? f.est_bytes - reuse : 0;
        const size_t freed = (sl.st && sl.frag != r->frag) ? sl.ctx->allocated : 0;
        if (s->budget && s->active > 0 && held - freed + need > s->budget) break;
        s->queue.pop_front();
        sl.req = r;
        r->slot = i;
        s->active += 1;
        held = held - freed + need;
        admitted.push_back(i);
      }
    }
    for (int i : admitted) {
      Slot& sl = s->slots[i];
      mps_status rc = start(s, sl);
      if (rc != MPS_OK) fail(s, sl, rc);
    }
    // ---- one pass over the admitted evaluations
    bool progressed = false;
    for (Slot& sl : s->slots) {
      Request* r = sl.req;
      if (!r) continue;
      const Fragment& f = s->frags[r->frag];
      if (r->phase == kGates) {
        if (sl.chunks_in_flight == 2) {
          cudaEvent_t oldest = sl.chunk_ev[(sl.chunk_head + 2 - 2) % 2];
          if (cudaEventQuery(oldest) != cudaSuccess) continue;
          cudaGetLastError();
          sl.chunks_in_flight -= 1;
        }
        const int g0 = r->next_gate;
        const int cnt = std::min(kGatesPerTurn, f.circ->n_gates - g0);
        mps_status rc = MPS_OK;
        if (cnt > 0)
          rc = state_apply_device_gates(sl.st, sl.st->d_bound + g0, &f.circ->q[g0], &f.circ->arity[g0], cnt);
        if (rc == MPS_OK) {
          cudaEventRecord(sl.chunk_ev[sl.chunk_head], sl.ctx->stream);
          sl.chunk_head = (sl.chunk_head + 1) % 2;
          sl.chunks_in_flight = std::min(2, sl.chunks_in_flight + 1);
          r->next_gate = g0 + cnt;
          if (r->next_gate >= f.circ->n_gates) r->phase = kWaitGates;
          progressed = true;
        } else {
          fail(s, sl, rc);
        }
      } else if (r->phase == kWaitGates) {
        cudaError_t q = cudaStreamQuery(sl.ctx->stream);
        if (q == cudaErrorNotReady) continue;
        mps_status rc = q == cudaSuccess ? MPS_OK : cuda_fail(q, "serving: circuit");
        if (rc == MPS_OK) rc = ham_energy_async(sl.st, const_cast<mps_ham*>(f.ham), nullptr);
        if (rc == MPS_OK) {
          cudaError_t e = cudaMemcpyAsync(sl.h_energy, sl.st->d_energy, sizeof(double), cudaMemcpyDeviceToHost,
                                          sl.ctx->stream);
          if (e == cudaSuccess)  // the status flags land in the second half of the pinned buffer
            e = cudaMemcpyAsync(sl.h_energy + 1, &sl.st->d_rep->not_converged, sizeof(StateFlags),
                                cudaMemcpyDeviceToHost, sl.ctx->stream);
          if (e != cudaSuccess) rc = cuda_fail(e, "serving: energy read-back");
        }
        if (rc == MPS_OK) {
          r->phase = kWaitEnergy;
          progressed = true;
        } else {
          fail(s, sl, rc);
        }
      } else if (r->phase == kWaitEnergy) {
        cudaError_t q = cudaStreamQuery(sl.ctx->stream);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) {
          fail(s, sl, cuda_fail(q, "serving: energy"));
          continue;
        }
        std::lock_guard<std::mutex> lk(s->mu);
        Fragment& fm = s->frags[r->frag];
        fm.est_bytes = std::max<size_t>(sl.ctx->allocated, 1);  // measured footprint from now on
        r->energy = *sl.h_energy;
        r->status = flags_status(*reinterpret_cast<const StateFlags*>(sl.h_energy + 1), true);
        if (r->status != MPS_OK) r->error = last_error();
        r->phase = kDone;
        r->latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - r->t_submit).count();
        sl.req = nullptr;
        s->active -= 1;
        s->completed += 1;
        s->peak_bytes = std::max(s->peak_bytes, slots_bytes(s));
        s->cv_done.notify_all();
        progressed = true;
      }
    }
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

}  // namespace
}  // namespace mpsv

using namespace mpsv;

extern "C" {

mps_status mps_server_create(int device, int32_t max_slots, size_t hbm_budget_bytes, mps_server** out) {
  if (!out || max_slots < 1 || max_slots > 256) {
    set_error("mps_server_create: out is NULL or max_slots = %d outside 1..256", max_slots);
    return MPS_EINVAL;
  }
  *out = nullptr;
  auto* s = new mps_server();
  s->device = device;
  s->max_slots = max_slots;
  s->budget = hbm_budget_bytes;
  s->slots.resize(max_slots);
  mps_status rc = MPS_OK;
  for (Slot& sl : s->slots) {
    if (rc == MPS_OK) rc = mps_ctx_create(device, nullptr, &sl.ctx);
    if (rc == MPS_OK) {
      DeviceGuard guard(device);
      cudaError_t e = cudaMallocHost(&sl.h_energy, 2 * sizeof(double));  // energy, then StateFlags
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.chunk_ev[0], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.chunk_ev[1], cudaEventDisableTiming);
      if (e != cudaSuccess) rc = cuda_fail(e, "mps_server_create");
    }
  }
  if (rc != MPS_OK) {
    for (Slot& sl : s->slots) {
      if (sl.h_energy) cudaFreeHost(sl.h_energy);
      for (cudaEvent_t e : sl.chunk_ev)
        if (e) cudaEventDestroy(e);
      if (sl.ctx) mps_ctx_destroy(sl.ctx);
    }
    delete s;
    return rc;
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return MPS_OK;
}

mps_status mps_server_add_fragment(mps_server* srv, const mps_circuit* circuit, const mps_ham* ham,
                                   const uint8_t* init_bits, const mps_config* cfg, int32_t* fragment_out) {
  if (!srv || !circuit || !ham || !cfg || !fragment_out) {
    set_error("mps_server_add_fragment: NULL argument");
    return MPS_EINVAL;
  }
  if (circuit->n != ham->n || circuit->ctx->device != srv->device || ham->ctx->device != srv->device) {
    set_error("mps_server_add_fragment: circuit (%d qubits) and Hamiltonian (%d) differ or are on another device",
              circuit->n, ham->n);
    return MPS_EINVAL;
  }
  if (cfg->chi_max < 1 || cfg->chi_max > 1024 || cfg->precision < MPS_PREC_FP64 || cfg->precision > MPS_PREC_AUTO) {
    set_error("mps_server_add_fragment: invalid mps_config (chi_max %d, precision %d)", cfg->chi_max, cfg->precision);
    return MPS_EINVAL;
  }
  Fragment f;
  f.circ = circuit;
  f.ham = ham;
  f.bits.assign(ham->n, 0);
  if (init_bits)
    for (int i = 0; i < ham->n; ++i) {
      if (init_bits[i] > 1) {
        set_error("mps_server_add_fragment: init_bits[%d] = %d", i, (int)init_bits[i]);
        return MPS_EINVAL;
      }
      f.bits[i] = init_bits[i];
    }
  f.cfg = *cfg;
  f.est_bytes = estimate_bytes(f);
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->frags.push_back(f);
  *fragment_out = (int32_t)srv->frags.size() - 1;
  return MPS_OK;
}

mps_status vqe_submit(mps_server* srv, int32_t fragment, const double* theta, uint64_t* ticket_out) {
  if (!srv || !ticket_out) {
    set_error("vqe_submit: NULL argument");
    return MPS_EINVAL;
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  if (fragment < 0 || fragment >= (int32_t)srv->frags.size()) {
    set_error("vqe_submit: unknown fragment %d", fragment);
    return MPS_EINVAL;
  }
  const Fragment& f = srv->frags[fragment];
  if (f.circ->n_params && !theta) {
    set_error("vqe_submit: theta is NULL");
    return MPS_EINVAL;
  }
  if (srv->stop) {
    set_error("vqe_submit: server is shutting down");
    return MPS_ESTATE;
  }
  if (srv->queue.size() >= kMaxQueue) {
    set_error("vqe_submit: %zu requests queued", srv->queue.size());
    return MPS_EBUSY;
  }
  auto* r = new Request();
  r->ticket = srv->next_ticket++;
  r->frag = fragment;
  r->theta.assign(theta, theta + f.circ->n_params);
  r->t_submit = Clock::now();
  srv->live[r->ticket] = r;
  srv->queue.push_back(r);
  *ticket_out = r->ticket;
  srv->cv_work.notify_one();
  return MPS_OK;
}

mps_status vqe_poll(mps_server* srv, uint64_t ticket, int32_t timeout_ms, double* energy_out, double* latency_ms_out) {
  if (!srv) {
    set_error("vqe_poll: NULL server");
    return MPS_EINVAL;
  }
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->live.find(ticket);
  if (it == srv->live.end()) {
    set_error("vqe_poll: unknown ticket %llu", (unsigned long long)ticket);
    return MPS_EINVAL;
  }
  Request* r = it->second;
  auto done = [&] { return r->phase == kDone; };
  if (timeout_ms < 0)
    srv->cv_done.wait(lk, done);
  else if (timeout_ms > 0)
    srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done);
  if (!done()) {
    set_error("vqe_poll: ticket %llu not finished", (unsigned long long)ticket);
    return MPS_ETIMEOUT;
  }
  const mps_status rc = r->status;
  if (energy_out) *energy_out = r->energy;
  if (latency_ms_out) *latency_ms_out = r->latency_ms;
  if (rc != MPS_OK) set_error("%s", r->error.c_str());
  srv->live.erase(it);
  delete r;
  return rc;
}

mps_status mps_server_stats(mps_server* srv, int64_t* completed_out, int32_t* active_out, int32_t* queued_out,
                            size_t* bytes_out, size_t* peak_bytes_out) {
  if (!srv) {
    set_error("mps_server_stats: NULL server");
    return MPS_EINVAL;
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  if (completed_out) *completed_out = srv->completed;
  if (active_out) *active_out = srv->active;
  if (queued_out) *queued_out = (int32_t)srv->queue.size();
  const size_t b = slots_bytes(srv);
  if (bytes_out) *bytes_out = b;
  if (peak_bytes_out) *peak_bytes_out = std::max(srv->peak_bytes, b);
  return MPS_OK;
}

void mps_server_destroy(mps_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    srv->cv_work.notify_all();
  }
  if (srv->worker.joinable()) srv->worker.join();
  DeviceGuard guard(srv->device);
  for (Slot& sl : srv->slots) {
    if (sl.st) mps_destroy(sl.st);
    if (sl.h_energy) cudaFreeHost(sl.h_energy);
    for (cudaEvent_t e : sl.chunk_ev)
      if (e) cudaEventDestroy(e);
    if (sl.ctx) mps_ctx_destroy(sl.ctx);
  }
  for (auto& kv : srv->live) delete kv.second;
  delete srv;
}

}  // extern "C"
