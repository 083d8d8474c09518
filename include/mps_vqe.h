/*
 * mps_vqe.h - C-ABI of the GB300 (sm_103a) MPS circuit simulator and
 * Pauli-sum energy of arXiv:2303.03681 ("Towards practical and massively
 * parallel quantum computing emulation for quantum chemistry").
 *
 * The library (libmpsvqe.so) keeps a matrix product state in right-canonical
 * form on one GPU and applies one- and two-qubit gates to it with the
 * Hastings update and SVD truncation (Methods, "MPS algorithm for quantum
 * circuit simulation": Eqs. mps, rightcanonicalcondition, tildeC, svdtildeC,
 * Bl), and evaluates E = sum_k c_k <psi|P_k|psi> over Pauli strings by
 * Eqs. expec1/expec2 (Methods, "The implementation of UCCSD with matrix
 * produce states"), sharing left environments between strings with a common
 * prefix.
 *
 * Conventions (all calls):
 *  - Sites are qubits 0..n-1.  Site tensor B_n has shape
 *    [chi_{n-1}][2][chi_n] (row-major).  Bond b sits left of site b
 *    (b = 0..n, chi_0 = chi_n = 1) and carries the singular values lam_b.
 *  - A two-qubit gate acts on adjacent sites (q, q+1); its 4x4 matrix is
 *    indexed by 2*i_q + i_{q+1} (site q is the more significant bit).  A
 *    statevector index has qubit 0 as its most significant bit.
 *  - Complex numbers in host arrays are (re, im) pairs of doubles.
 *  - Host arrays passed in are read during the call and stay owned by the
 *    caller.  Handles are owned by the library until the matching *_destroy.
 *  - Every call returns an mps_status and never aborts the process; the
 *    message of the last failure on the calling thread is mps_last_error().
 *  - Work is issued on the context's CUDA stream.  Calls that return host
 *    results synchronise that stream; calls named *_async do not.
 *  - Calls on one context are not thread-safe; different contexts are.
 */
#ifndef MPS_VQE_H
#define MPS_VQE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MPS_OK = 0,
  MPS_EINVAL = 1,     /* bad argument (null handle, non-adjacent gate, size) */
  MPS_ENOMEM = 2,     /* device allocation failed or the allocation cap was hit */
  MPS_ECUDA = 3,      /* a CUDA runtime call failed */
  MPS_ETIMEOUT = 4,   /* a bounded device-side wait ran out */
  MPS_ENOTCONV = 5,   /* a truncation SVD reached its Jacobi sweep cap (Algorithm 1's
                         stopping test was not met).  The result is still delivered: the
                         state is updated and the energy written with that SVD as it stood,
                         and the state stays usable.  Counted in
                         mps_report.svd_not_converged.  Returned by mps_apply_gates,
                         vqe_eval, vqe_eval_batch (per request) and vqe_poll. */
  MPS_EBUSY = 6,      /* serving queue full */
  MPS_ESTATE = 7      /* state left inconsistent by an earlier failure: reset it */
} mps_status;

/* Arithmetic of a state.  The truncation SVD is FP64-accurate and the energy
 * sum FP64 in every mode unless mps_config.svd_fp64 = 0.  MPS_PREC_FP64
 * stores complex128; its CUDA-core contractions (theta, B~_q, environments)
 * and the FP64-accurate Jacobi sweeps compute in double-float arithmetic
 * (pairs of FP32 values, about 2^-46 relative per operation) on the FP32
 * units, since this part executes FP64 at 1/64 of the FP32 rate; results
 * are stored as complex128.  The split-product modes keep
 * complex64 storage and run the theta contraction C = Q (B_q B_{q+1}) and
 * B~_q = C V^dagger (Eqs. tildeC, Bl) as tensor-core GEMMs (tcgen05, operands
 * loaded with TMA) in which every real operand value is split into two
 * pieces and each real product is the sum of three piece products
 * (hi*hi + hi*lo + lo*hi) accumulated in FP32; their environment
 * contractions use the tensor cores at bond dimension >= 64 as
 * mps_config.tensor_cores does. */
typedef enum {
  MPS_PREC_FP64 = 0,   /* complex128 storage, double-float contractions */
  MPS_PREC_FP32 = 1,   /* complex64 storage, FP32 CUDA-core contractions */
  MPS_PREC_BF16X3 = 2, /* complex64 storage, BF16 pieces (16 bits of each value kept) */
  MPS_PREC_TF32X3 = 3, /* complex64 storage, TF32 pieces (22 bits kept: about FP32 accuracy) */
  MPS_PREC_AUTO = 4    /* complex64 storage, TF32X3 where a bond capacity reaches 256, FP32
                          CUDA cores below */
} mps_precision;

typedef struct {
  int32_t chi_max;        /* bond-dimension cap (>= 1) */
  int32_t precision;      /* mps_precision */
  double trunc_rel;       /* keep s_i > trunc_rel * s_1 (0: keep all nonzero) */
  int32_t svd_fp64;       /* 0: Jacobi SVD in the storage precision;
                             1: FP64-accurate Jacobi SVD (thetas whose column capacity is 32 or
                                more: FP32 sweeps to FP32 convergence, two FP64
                                re-orthonormalisation passes of V, A = C~ V rebuilt in FP64,
                                double-float sweeps on the FP32 units to a stopping rule at unit
                                roundoff 2^-46; smaller thetas: every sweep in FP64);
                             2: every Jacobi sweep in FP64 */
  int32_t svd_max_sweeps; /* Jacobi sweep cap; 0 selects 60 */
  double svd_tol;         /* rotate a pair while |b_ij| > tol sqrt(b_ii b_jj); 0: default */
  int32_t tensor_cores;   /* complex64 states: 1 = environment contractions on the tensor
                             cores (tcgen05, TF32 hi/lo split, 4 products, FP32 accumulation);
                             0 = FP32 CUDA-core kernels.  Ignored for complex128. */
} mps_config;

/* One gate.  arity 1: u holds the 2x2 matrix (4 complex = 8 doubles, row
 * major); arity 2: the 4x4 matrix (16 complex = 32 doubles).  A two-qubit
 * gate acts on (q, q+1) and needs q + 1 < n. */
typedef struct {
  int32_t q;
  int32_t arity;
  double u[32];
} mps_gate;

/* One gate of a circuit template: G = exp(i phi) M_plus + exp(-i phi) M_minus
 * with phi = coeff * theta[param]; param = -1 marks a fixed gate (G = M_plus
 * + M_minus).  Matrix layout as in mps_gate. */
typedef struct {
  int32_t q;
  int32_t arity;
  int32_t param;
  int32_t reserved;
  double coeff;
  double m_plus[32];
  double m_minus[32];
} mps_template_gate;

/* Truncation statistics accumulated since the last reset. */
typedef struct {
  double discarded_weight;  /* sum over gates of 1 - sum(kept s^2) / sum(s^2) */
  double min_kept_sv;       /* smallest kept normalised singular value */
  int32_t max_chi;          /* largest bond dimension reached */
  int32_t degenerate_cuts;  /* cuts at chi_max inside a pair equal to 1e-10 */
  int32_t svd_not_converged;/* SVDs that hit the sweep cap */
  int32_t max_sweeps_used;  /* largest number of Jacobi sweeps of one SVD */
  int64_t two_qubit_gates;  /* two-qubit gates applied */
  double svd_flops;         /* real flops of the Jacobi sweeps run (dots + rotations) */
  int64_t svd_sweeps_fp32;  /* Jacobi sweeps run in FP32, summed over SVDs */
  int64_t svd_sweeps_fp64;  /* Jacobi sweeps run in FP64, summed over SVDs */
  double svd_phase_cycles[4]; /* SM clock cycles of the cluster SVDs (first CTA), summed: column
                                 load, FP32 sweeps, FP64 re-orthonormalisation of V and A = C~ V,
                                 FP64 sweeps with the truncation and output */
} mps_report;

/* Kernel classes for mps_ctx_profile_read. */
typedef enum {
  MPS_K_THETA = 0,     /* theta contraction + gate + lam scaling */
  MPS_K_SVD = 1,       /* Jacobi SVD + truncation */
  MPS_K_G3 = 2,        /* B~_q = C V^dagger */
  MPS_K_GATE1 = 3,     /* one-qubit gate */
  MPS_K_SETUP = 4,     /* reset, angle binding, fills */
  MPS_K_ENV_M = 5,     /* environment times site tensor */
  MPS_K_ENV_CHILD = 6, /* child environment */
  MPS_K_ENV_LEAF = 7,  /* leaf expectation values */
  MPS_K_ENV_TRACE = 8, /* trace expectation values */
  MPS_K_REDUCE = 9,    /* FP64 energy sum and observable row sums */
  MPS_K_COUNT = 10
} mps_kernel_kind;

typedef struct mps_ctx mps_ctx;
typedef struct mps_state mps_state;
typedef struct mps_ham mps_ham;
typedef struct mps_circuit mps_circuit;

/* Message of the last failed call on this thread ("" if none). */
const char* mps_last_error(void);

/* Library version string. */
const char* mps_version(void);

/* Create a context on CUDA device `device` issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = a new non-blocking stream owned by the context). */
mps_status mps_ctx_create(int device, void* cuda_stream, mps_ctx** out);
mps_status mps_ctx_synchronize(mps_ctx* ctx);
/* Cap on the device bytes this context may allocate (0 = no cap).  An
 * allocation beyond it fails with MPS_ENOMEM. */
mps_status mps_ctx_set_alloc_limit(mps_ctx* ctx, size_t bytes);
mps_status mps_ctx_bytes_allocated(const mps_ctx* ctx, size_t* out);
/* Destroys the context and frees its device memory.  Destroy its states,
 * Hamiltonians and circuits first: their handles become invalid. */
void mps_ctx_destroy(mps_ctx* ctx);
/* Circuit replay as CUDA graphs (default on).  With graphs on, the first
 * mps_apply_circuit_async / vqe_eval / vqe_eval_batch of a (state, circuit)
 * pair captures the bind kernel and every gate launch into a graph on the
 * context's stream; later calls copy theta in and replay the graph, so the
 * host issues one launch per circuit instead of three per gate.  A new
 * circuit, a grown theta workspace or a changed profiling mask re-captures.
 * enable = 0 launches every kernel from the host.  The results are the same
 * either way.  Returns MPS_EINVAL for a NULL context. */
mps_status mps_ctx_set_graphs(mps_ctx* ctx, int32_t enable);

/* Kernel timing: for every kernel class whose bit is set in `mask`
 * (bit k = mps_kernel_kind k) the library brackets each launch with CUDA
 * events on the context stream.  Launch counts are always kept. */
mps_status mps_ctx_profile(mps_ctx* ctx, uint32_t mask);
/* Launches of class `kind` and their summed device time (ms, timed launches
 * only) since the last reset; synchronises the stream.  reset != 0 clears. */
mps_status mps_ctx_profile_read(mps_ctx* ctx, int32_t kind, int64_t* launches, int64_t* timed_launches,
                                double* ms, int32_t reset);

/* Create an n-qubit MPS in the computational basis state |init_bits>
 * (init_bits: n bytes, 0/1; NULL = |0...0>) - the chi = 1 product state of
 * the paper's Hartree-Fock reference.  Device memory for every site is sized
 * for min(chi_max, 2^b, 2^(n-b)) on each bond. */
mps_status mps_create(mps_ctx* ctx, int32_t n_qubits, const uint8_t* init_bits,
                      const mps_config* cfg, mps_state** out);
/* Return the state to |init_bits> (NULL = |0...0>) and clear its report. */
mps_status mps_reset(mps_state* st, const uint8_t* init_bits);
void mps_destroy(mps_state* st);

/* Apply n gates in order (one-qubit: Methods single-qubit gate equation;
 * two-qubit: Hastings update of Eqs. tildeC, svdtildeC, Bl with truncation
 * to min(chi_max, #{s_i > trunc_rel s_1}) and renormalisation of the kept
 * singular values).  `report` (nullable) receives the accumulated
 * statistics; this call synchronises the stream.  MPS_ENOTCONV when an SVD
 * issued since the host last read the state's report (this call, or
 * asynchronous circuits before it; mps_reset clears the count) reached its
 * sweep cap: the gates are applied and the report is filled all the same. */
mps_status mps_apply_gates(mps_state* st, const mps_gate* gates, size_t n, mps_report* report);

/* The theta contraction of one two-qubit gate on its own (the G1 step of the
 * Hastings update, Methods "MPS algorithm for quantum circuit simulation":
 * C = Q (B_q B_{q+1}) before the lam scaling of Eq. tildeC), for complex64
 * site tensors in device memory:
 *   B_left   [chi_l][2][chi_m] complex64 (interleaved re, im floats);
 *   B_right  [chi_m][2][chi_r] complex64;
 *   gate     host array, 4x4 row-major complex (32 doubles), index 2 i_q + i_{q+1};
 *   C_out    [(a_l, i)][(j, a_r)] = (2 chi_l) x (2 chi_r) complex64, row-major,
 *            C_out[(2 a_l + i) * 2 chi_r + j chi_r + a_r].
 * precision: MPS_PREC_FP32 (CUDA cores, FP32), MPS_PREC_TF32X3 or
 * MPS_PREC_BF16X3 (the tensor-core split products mps_apply_gates uses for
 * such states); others fail with MPS_EINVAL, as do bond dimensions outside
 * 1..4096.  Work is issued on the context stream and the call returns without
 * synchronising (the host arrays are copied before it returns); the context
 * keeps a workspace sized for the largest call so far (released with the
 * context).  The device arrays belong to the caller and must not overlap. */
mps_status mps_contract_theta(mps_ctx* ctx, int32_t precision, int32_t chi_l, int32_t chi_m, int32_t chi_r,
                              const void* B_left, const void* B_right, const double* gate, void* C_out);

/* The truncation SVD of one theta on its own (the S1/S2 step of the Hastings
 * update: one-sided Jacobi SVD of Algorithm 1, Methods "SVD and one-side
 * jacobi", then the truncation rule of mps_apply_gates).  C is an m x n
 * complex matrix in device memory, row-major (complex128 for MPS_PREC_FP64,
 * complex64 for MPS_PREC_FP32); m and n must be even (m = 2 chi_l, n =
 * 2 chi_r in the gate update) and in 2..4096.  The kept count k =
 * min(chi_max, #{s_i > trunc_rel s_1}) >= 1 goes to *k_out (host); s_out
 * (device, room for min(m, n) doubles) receives s_1 >= ... >= s_k, not
 * renormalised; Vh_out (device, room for min(chi_max, m, n) x n entries of the
 * input precision, row-major) the rows of V^H, i.e. the right singular
 * vectors conjugated.  svd_fp64 as in mps_config.  `report` (nullable)
 * receives the sweep counts and the discarded weight.  The context keeps a
 * workspace sized for the largest call so far; the call synchronises its
 * stream and returns MPS_ENOTCONV (results written) when the sweep cap was
 * reached. */
mps_status mps_truncated_svd(mps_ctx* ctx, int32_t precision, int32_t m, int32_t n, const void* C, int32_t chi_max,
                             double trunc_rel, int32_t svd_fp64, double* s_out, void* Vh_out, int32_t* k_out,
                             mps_report* report);

/* Upload a circuit template (see mps_template_gate) with n_params angles. */
mps_status mps_circuit_create(mps_ctx* ctx, int32_t n_qubits, const mps_template_gate* gates,
                              size_t n_gates, int32_t n_params, mps_circuit** out);
void mps_circuit_destroy(mps_circuit* c);
/* Bind theta (host array of n_params doubles, or a device pointer when
 * theta_on_device != 0) and apply the circuit without synchronising. */
mps_status mps_apply_circuit_async(mps_state* st, const mps_circuit* c, const double* theta,
                                   int theta_on_device);

/* Upload a Hamiltonian sum_k coeffs[k] P_k: ops is n_terms x n_qubits bytes
 * (0=I 1=X 2=Y 3=Z), coeffs real.  The strings are arranged on the host in
 * a prefix trie (first non-identity site, then the operators left to right)
 * whose nodes are the shared left environments of Eq. expec2. */
mps_status mps_hamiltonian_create(mps_ctx* ctx, int32_t n_qubits, size_t n_terms,
                                  const uint8_t* ops, const double* coeffs, mps_ham** out);
/* Trie statistics: n_nodes materialised environments, n_levels sites. */
mps_status mps_hamiltonian_info(const mps_ham* h, int64_t* n_terms, int64_t* n_nodes,
                                int64_t* max_level_nodes);
void mps_ham_destroy(mps_ham* h);

/* E = sum_k c_k <P_k> in FP64 (Eq. expec2 per string: lam^2 of the bond left
 * of the first non-identity site, transfer products to the last one, trace);
 * norm_out (nullable) gets sum(lam_1^2) of the first bond.  Synchronises. */
mps_status mps_energy(mps_state* st, const mps_ham* h, double* energy_out, double* norm_out);
/* Same, writing the energy to device memory without synchronising. */
mps_status mps_energy_async(mps_state* st, const mps_ham* h, double* d_energy_out);
/* Per-term expectation values <P_k> (host array of n_terms doubles). */
mps_status mps_expectations(mps_state* st, const mps_ham* h, double* values_out);

/* Linear observables of one string set: the reduced density matrices of the
 * paper's Methods, "The DMET method" (1-RDM <a+_p a_q>, 2-RDM
 * <a+_p a+_q a_r a_s>, from which the fragment energy and electron count
 * follow).  Under the Jordan-Wigner map every RDM element is a complex
 * combination of Pauli strings, so all of them follow from the per-string
 * values <P_j> (Eq. expec2, environments shared through the trie of the
 * string set):
 *   values[r] = sum_{e = row_ptr[r]}^{row_ptr[r+1]-1} weights[e] <P_{cols[e]}>.
 * `strings` is a Hamiltonian handle whose terms are the strings P_j (its
 * coefficients are not used); it must outlive the observables handle, which
 * lives in its context.  row_ptr: n_rows + 1 int64, row_ptr[0] = 0,
 * non-decreasing; cols: row_ptr[n_rows] int32 in [0, n_terms); weights:
 * 2 * row_ptr[n_rows] doubles (re, im), finite.  All host arrays, copied
 * during the call.  MPS_EINVAL for NULL or inconsistent arguments (no handle
 * is created; *out = NULL), MPS_ENOMEM / MPS_ECUDA from the upload. */
typedef struct mps_obs mps_obs;
mps_status mps_observables_create(const mps_ham* strings, size_t n_rows, const int64_t* row_ptr,
                                  const int32_t* cols, const double* weights, mps_obs** out);
/* Evaluate every row for the state's current MPS: values_out is a host array
 * of 2 * n_rows doubles (re, im).  The per-string values come from the
 * energy kernels; the row sums run on the device in FP64 in a fixed order
 * (one launch).  The state keeps an output buffer of n_rows entries between
 * calls.  Synchronises the state's stream; MPS_EINVAL if the string set has
 * another qubit count or device than the state. */
mps_status mps_observables_eval(mps_state* st, const mps_obs* obs, double* values_out);
void mps_observables_destroy(mps_obs* obs);

/* Bond dimensions chi_0..chi_n (host array of n+1 int32). */
mps_status mps_bond_dims(mps_state* st, int32_t* chi_out);
/* Host copy of the state: tensors_out receives every B_n (row-major
 * [chi_{n-1}][2][chi_n], complex128 as (re, im)) back to back; lam_out every
 * lam_b, b = 0..n, back to back.  Sizes follow mps_bond_dims. */
mps_status mps_export(mps_state* st, double* tensors_out, size_t tensors_cap_doubles, double* lam_out,
                      size_t lam_cap);
mps_status mps_get_report(mps_state* st, mps_report* out);

/* One VQE energy evaluation per request: reset to init_bits, apply the
 * template bound to theta, evaluate the Hamiltonian.  Requests run in order
 * on the context stream; energies_out[i] (host) and status_out[i]
 * (nullable) receive the results.  theta and init_bits are host arrays.
 * A request whose circuit had an SVD reach its sweep cap gets MPS_ENOTCONV
 * with its energy written; other failures write 0.  The return value is the
 * first status that is not MPS_OK. */
typedef struct {
  mps_state* state;
  const mps_circuit* circuit;
  const mps_ham* ham;
  const double* theta;
  const uint8_t* init_bits;
} vqe_request;
mps_status vqe_eval(mps_ctx* ctx, const vqe_request* reqs, size_t n, double* energies_out,
                    mps_status* status_out);

/* Batched form of vqe_eval (the fragment-level parallelism of the paper's
 * Methods, "Heterogeneous parallelization strategy", on one GPU): the
 * requests may belong to different contexts, each with its own stream, and
 * must use distinct states.  Requests are grouped by context; up to 16 host
 * threads issue the groups' gates, each going round-robin over its requests
 * (gate g of every request before gate g+1), so independent evaluations
 * overlap on the device; then the calling thread evaluates each energy.
 * Streams beyond the device's hardware work queues are serialised by the
 * driver: set CUDA_DEVICE_MAX_CONNECTIONS (up to 32) to at least the number
 * of contexts before the process creates its CUDA context.
 * energies_out[i] / status_out[i] (host, status nullable) as in vqe_eval
 * (MPS_ENOTCONV included); the return value is the first status that is not
 * MPS_OK. */
mps_status vqe_eval_batch(const vqe_request* reqs, size_t n, double* energies_out, mps_status* status_out);
/* Same with device-resident data: every request's theta is a device pointer
 * and d_energies_out is a device array of n doubles.  The call returns once
 * all work is issued (each energy reads its state's bond dimensions, which
 * waits for that state's circuit); synchronise the streams before reading.
 * Sweep-cap hits are not reported here (the call returns before the SVDs
 * run): read mps_report.svd_not_converged of each state afterwards. */
mps_status vqe_eval_batch_async(const vqe_request* reqs, size_t n, double* d_energies_out, mps_status* status_out);

/* ---- serving: continuous batching of energy evaluations -----------------
 *
 * A server owns up to max_slots evaluation slots on one device, each with its
 * own stream and state.  Fragments (circuit template + Hamiltonian + reference
 * state + mps_config) are registered once and stay resident.  vqe_submit
 * queues E(theta) for a fragment and returns at once; a native worker thread
 * admits queued requests into free slots while the device memory the server
 * has allocated plus the request's estimated footprint stays within
 * hbm_budget_bytes (0 = no budget), issues every admitted evaluation's gates
 * a few at a time in turn (requests arriving while others run join between
 * gate groups), evaluates its energy and completes it.  This is the paper's
 * fragment-level parallelism (Methods, "Heterogeneous parallelization
 * strategy") mapped to one GPU.  The result of a
 * request does not depend on what else is in flight: the same kernels run on
 * the same data.  Handles passed to a server (circuit, Hamiltonian) must
 * outlive it. */
typedef struct mps_server mps_server;

mps_status mps_server_create(int device, int32_t max_slots, size_t hbm_budget_bytes, mps_server** out);
/* Register a resident fragment; init_bits: n bytes (NULL = |0...0>). */
mps_status mps_server_add_fragment(mps_server* srv, const mps_circuit* circuit, const mps_ham* ham,
                                   const uint8_t* init_bits, const mps_config* cfg, int32_t* fragment_out);
/* Queue E(theta) for a fragment (theta: host, copied); MPS_EBUSY when the
 * queue holds max_queue requests already. */
mps_status vqe_submit(mps_server* srv, int32_t fragment, const double* theta, uint64_t* ticket_out);
/* Wait up to timeout_ms (0 = do not wait, < 0 = forever) for a request.
 * Returns MPS_OK with the energy and the submit-to-completion latency in
 * milliseconds (MPS_ENOTCONV with both when an SVD of the evaluation reached
 * its sweep cap), MPS_ETIMEOUT if it is not done yet, MPS_EINVAL for an
 * unknown ticket, or the request's own failure status.  A completed ticket is
 * released by the poll that returns it. */
mps_status vqe_poll(mps_server* srv, uint64_t ticket, int32_t timeout_ms, double* energy_out, double* latency_ms_out);
/* Counters: requests completed, currently admitted, queued; device bytes the
 * server holds (its high-water mark in peak_bytes_out). */
mps_status mps_server_stats(mps_server* srv, int64_t* completed_out, int32_t* active_out, int32_t* queued_out,
                            size_t* bytes_out, size_t* peak_bytes_out);
/* Stops the worker after the requests in flight finish and frees the slots. */
void mps_server_destroy(mps_server* srv);

/* Apply one two-qubit gate to two adjacent site tensors that live in the
 * caller's device memory, allocating nothing.
 *
 * The paper has no counterpart to this call.  It exists for callers that
 * cannot allocate device memory: code running in a CUDA host callback or a
 * stream-ordered host function (where allocating CUDA calls are not allowed),
 * embedders that give the library a fixed, pre-partitioned share of device
 * memory, and processes whose memory budget was fixed at start-up.  The
 * gate's scratch (theta, the Jacobi matrices, the bond dimensions and the
 * truncation report) lives in one fixed array of 197,632 bytes compiled into
 * the library, which every GPU that loads the library keeps until the
 * process exits.
 *
 * Arguments (device pointers unless noted; complex128 as (re, im) doubles):
 *   device, cuda_stream  the device whose memory the pointers refer to and
 *                        the stream to issue on (NULL = legacy default);
 *   chi_l, chi_m, chi_r  current bond dimensions left of site q, between q
 *                        and q+1, right of q+1; chi_l, chi_r <= 32 and
 *                        chi_m <= 64 (larger sizes fail with MPS_EINVAL);
 *   B_left   [chi_l][2][chi_m] on entry, [chi_l][2][k] on return; room for
 *            chi_l*2*max(chi_m, kmax) entries, kmax = min(chi_max, 2 chi_l, 2 chi_r);
 *   B_right  [chi_m][2][chi_r] on entry, [k][2][chi_r] on return; room for
 *            max(chi_m, kmax)*2*chi_r entries;
 *   lam_left chi_l singular values of the bond left of site q;
 *   lam_out  receives the k new singular values (room for kmax);
 *   gate     host array, 4x4 row-major complex (32 doubles), index 2 i_q + i_{q+1};
 *   chi_max, trunc_rel  truncation as in mps_config;
 *   chi_out  receives k (one int32).
 * The update is the one mps_apply_gates makes for a complex128 state, except
 * that SVD convergence is not reported: the call returns before the work
 * runs, and an SVD that reaches the sweep cap (60 sweeps) is written as it
 * stands.  The call returns after issuing the work; synchronise the stream
 * before reading the outputs.  MPS_EINVAL for a device that does not exist
 * (checked before anything is issued or cached).  The first call on each device sets the library up for that
 * device (it looks up the scratch array's device address); make it before
 * any stream capture.  All calls share the scratch array and it keeps the
 * last call's contents (the kernels overwrite what they read): calls whose
 * work overlaps on the GPU, from several streams or threads, race on it. */
mps_status mps_gate2_noalloc(int device, void* cuda_stream, int32_t chi_l, int32_t chi_m, int32_t chi_r,
                             double* B_left, double* B_right, const double* lam_left, double* lam_out,
                             const double* gate, int32_t chi_max, double trunc_rel, int32_t* chi_out);

#ifdef __cplusplus
}
#endif

#endif /* MPS_VQE_H */
