"""Python binding of the C-ABI in include/mps_vqe.h (argument marshalling only).

Every operation runs in libmpsvqe.so on the GPU; there is no Python or CPU
fallback.  Importing this module loads the library and raises if it is
missing or cannot be loaded.
"""

import atexit
import ctypes
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpsvqe.so")

MPS_OK, MPS_EINVAL, MPS_ENOMEM, MPS_ECUDA, MPS_ETIMEOUT, MPS_ENOTCONV, MPS_EBUSY, MPS_ESTATE = range(8)
STATUS_NAMES = ["MPS_OK", "MPS_EINVAL", "MPS_ENOMEM", "MPS_ECUDA", "MPS_ETIMEOUT", "MPS_ENOTCONV", "MPS_EBUSY",
                "MPS_ESTATE"]
PRECISIONS = {"fp64": 0, "fp32": 1, "bf16x3": 2, "tf32x3": 3, "auto": 4}
KERNEL_KINDS = ["theta", "svd", "g3", "gate1", "setup", "env_m", "env_child", "env_leaf", "env_trace", "reduce"]

# numpy views of the C structs (layouts match include/mps_vqe.h on LP64 hosts)
GATE_DTYPE = np.dtype([("q", "<i4"), ("arity", "<i4"), ("u", "<f8", (32,))])
TEMPLATE_GATE_DTYPE = np.dtype([("q", "<i4"), ("arity", "<i4"), ("param", "<i4"), ("reserved", "<i4"),
                                ("coeff", "<f8"), ("m_plus", "<f8", (32,)), ("m_minus", "<f8", (32,))])
assert GATE_DTYPE.itemsize == 264 and TEMPLATE_GATE_DTYPE.itemsize == 536


class MpsError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {message}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("chi_max", ctypes.c_int32), ("precision", ctypes.c_int32), ("trunc_rel", ctypes.c_double),
                ("svd_fp64", ctypes.c_int32), ("svd_max_sweeps", ctypes.c_int32), ("svd_tol", ctypes.c_double),
                ("tensor_cores", ctypes.c_int32)]


class Report(ctypes.Structure):
    _fields_ = [("discarded_weight", ctypes.c_double), ("min_kept_sv", ctypes.c_double),
                ("max_chi", ctypes.c_int32), ("degenerate_cuts", ctypes.c_int32),
                ("svd_not_converged", ctypes.c_int32), ("max_sweeps_used", ctypes.c_int32),
                ("two_qubit_gates", ctypes.c_int64), ("svd_flops", ctypes.c_double),
                ("svd_sweeps_fp32", ctypes.c_int64), ("svd_sweeps_fp64", ctypes.c_int64),
                ("svd_phase_cycles", ctypes.c_double * 4)]

    def as_dict(self):
        return {k: (list(getattr(self, k)) if k == "svd_phase_cycles" else getattr(self, k)) for k, _ in self._fields_}


class VqeRequest(ctypes.Structure):
    _fields_ = [("state", ctypes.c_void_p), ("circuit", ctypes.c_void_p), ("ham", ctypes.c_void_p),
                ("theta", ctypes.c_void_p), ("init_bits", ctypes.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; "
                           f"g.build()\"` (needs nvcc for sm_103a)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, SZ, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t, ctypes.c_double
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "mps_last_error": ([], ctypes.c_char_p),
        "mps_version": ([], ctypes.c_char_p),
        "mps_ctx_create": ([ctypes.c_int, P, PP], ctypes.c_int),
        "mps_ctx_synchronize": ([P], ctypes.c_int),
        "mps_ctx_set_alloc_limit": ([P, SZ], ctypes.c_int),
        "mps_ctx_bytes_allocated": ([P, ctypes.POINTER(SZ)], ctypes.c_int),
        "mps_ctx_destroy": ([P], None),
        "mps_create": ([P, I32, P, ctypes.POINTER(Config), PP], ctypes.c_int),
        "mps_reset": ([P, P], ctypes.c_int),
        "mps_destroy": ([P], None),
        "mps_apply_gates": ([P, P, SZ, ctypes.POINTER(Report)], ctypes.c_int),
        "mps_circuit_create": ([P, I32, P, SZ, I32, PP], ctypes.c_int),
        "mps_circuit_destroy": ([P], None),
        "mps_apply_circuit_async": ([P, P, P, ctypes.c_int], ctypes.c_int),
        "mps_hamiltonian_create": ([P, I32, SZ, P, P, PP], ctypes.c_int),
        "mps_hamiltonian_info": ([P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                  ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "mps_ham_destroy": ([P], None),
        "mps_energy": ([P, P, ctypes.POINTER(D), ctypes.POINTER(D)], ctypes.c_int),
        "mps_energy_async": ([P, P, P], ctypes.c_int),
        "mps_expectations": ([P, P, P], ctypes.c_int),
        "mps_observables_create": ([P, SZ, P, P, P, PP], ctypes.c_int),
        "mps_observables_eval": ([P, P, P], ctypes.c_int),
        "mps_observables_destroy": ([P], None),
        "mps_bond_dims": ([P, P], ctypes.c_int),
        "mps_export": ([P, P, SZ, P, SZ], ctypes.c_int),
        "mps_get_report": ([P, ctypes.POINTER(Report)], ctypes.c_int),
        "vqe_eval": ([P, P, SZ, P, P], ctypes.c_int),
        "vqe_eval_batch": ([P, SZ, P, P], ctypes.c_int),
        "vqe_eval_batch_async": ([P, SZ, P, P], ctypes.c_int),
        "mps_server_create": ([ctypes.c_int, I32, SZ, PP], ctypes.c_int),
        "mps_server_add_fragment": ([P, P, P, P, ctypes.POINTER(Config), ctypes.POINTER(I32)], ctypes.c_int),
        "vqe_submit": ([P, I32, P, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "vqe_poll": ([P, ctypes.c_uint64, I32, ctypes.POINTER(D), ctypes.POINTER(D)], ctypes.c_int),
        "mps_server_stats": ([P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(I32), ctypes.POINTER(I32),
                              ctypes.POINTER(SZ), ctypes.POINTER(SZ)], ctypes.c_int),
        "mps_server_destroy": ([P], None),
        "mps_ctx_profile": ([P, ctypes.c_uint32], ctypes.c_int),
        "mps_ctx_set_graphs": ([P, I32], ctypes.c_int),
        "mps_contract_theta": ([P, I32, I32, I32, I32, P, P, P, P], ctypes.c_int),
        "mps_truncated_svd": ([P, I32, I32, I32, P, I32, D, I32, P, P, ctypes.POINTER(I32), ctypes.POINTER(Report)],
                              ctypes.c_int),
        "mps_ctx_profile_read": ([P, I32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                  ctypes.POINTER(D), I32], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()


def library():
    return _lib


def _check(status):
    if status != MPS_OK:
        raise MpsError(status, _lib.mps_last_error().decode())


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def version() -> str:
    return _lib.mps_version().decode()


# ---------------------------------------------------------------------------
# marshalling of generator objects
# ---------------------------------------------------------------------------

def _pack_matrices(u, arity):
    """(G, 4, 4) complex -> (G, 32) doubles: 4x4 row-major, or 2x2 first."""
    g = u.shape[0]
    out = np.zeros((g, 32))
    two = arity == 2
    m4 = np.ascontiguousarray(u[two]).reshape(-1, 16)
    out[two] = np.stack([m4.real, m4.imag], axis=-1).reshape(-1, 32)
    m2 = np.ascontiguousarray(u[~two][:, :2, :2]).reshape(-1, 4)
    out[~two, :8] = np.stack([m2.real, m2.imag], axis=-1).reshape(-1, 8)
    return out


def gates_to_abi(gates) -> np.ndarray:
    """GateList -> array of mps_gate."""
    arr = np.zeros(gates.n_gates, dtype=GATE_DTYPE)
    arr["q"] = gates.q
    arr["arity"] = gates.arity
    arr["u"] = _pack_matrices(np.asarray(gates.u), np.asarray(gates.arity))
    return arr


def template_to_abi(tmpl) -> np.ndarray:
    """CircuitTemplate -> array of mps_template_gate."""
    arr = np.zeros(tmpl.n_gates, dtype=TEMPLATE_GATE_DTYPE)
    arr["q"] = tmpl.q
    arr["arity"] = tmpl.arity
    arr["param"] = tmpl.param
    arr["coeff"] = tmpl.coeff
    arr["m_plus"] = _pack_matrices(tmpl.m_plus, tmpl.arity)
    arr["m_minus"] = _pack_matrices(tmpl.m_minus, tmpl.arity)
    return arr


# ---------------------------------------------------------------------------
# handles
# ---------------------------------------------------------------------------
#
# A context owns the device memory of its states, Hamiltonians and circuits.
# Children are released before their context whatever order Python finalises
# them in (at interpreter exit reference cycles are collected in arbitrary
# order): Context.close() closes its live children first, and a child whose
# context is already closed only drops its handle.

_live_contexts = weakref.WeakSet()


_live_servers = weakref.WeakSet()


@atexit.register
def _close_all_contexts():
    for srv in list(_live_servers):  # servers use circuits and Hamiltonians of contexts
        try:
            srv.close()
        except Exception:
            pass
    for c in list(_live_contexts):
        try:
            c.close()
        except Exception:
            pass


class _Child:
    handle = None
    _destroy = None

    def _adopt(self, ctx):
        self.ctx = ctx
        ctx._children.add(self)

    def close(self):
        if self.handle:
            if self.ctx.handle:
                type(self)._destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """A device and the CUDA stream the library issues its work on.

    ``stream`` may be a torch.cuda.Stream, an integer cudaStream_t or None (a
    private non-blocking stream)."""

    def __init__(self, device: int = 0, stream=None):
        handle = ctypes.c_void_p()
        s = None
        if stream is not None:
            s = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        _check(_lib.mps_ctx_create(int(device), s, ctypes.byref(handle)))
        self.handle = handle
        self.device = device
        self._stream = stream
        self._children = weakref.WeakSet()
        _live_contexts.add(self)

    def synchronize(self):
        _check(_lib.mps_ctx_synchronize(self.handle))

    def set_alloc_limit(self, nbytes: int):
        _check(_lib.mps_ctx_set_alloc_limit(self.handle, int(nbytes)))

    def set_graphs(self, enable: bool):
        """Replay circuits as CUDA graphs (default) or launch every kernel from the host."""
        _check(_lib.mps_ctx_set_graphs(self.handle, 1 if enable else 0))

    def profile(self, kinds=()):
        """Time every launch of the named kernel classes with CUDA events."""
        mask = 0
        for k in kinds:
            mask |= 1 << KERNEL_KINDS.index(k)
        _check(_lib.mps_ctx_profile(self.handle, mask))

    def profile_read(self, reset: bool = False) -> dict:
        """{kind: (launches, timed launches, ms)} since the last reset."""
        out = {}
        for i, k in enumerate(KERNEL_KINDS):
            a, b, ms = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
            _check(_lib.mps_ctx_profile_read(self.handle, i, ctypes.byref(a), ctypes.byref(b), ctypes.byref(ms),
                                             1 if reset else 0))
            out[k] = (a.value, b.value, ms.value)
        return out

    def bytes_allocated(self) -> int:
        v = ctypes.c_size_t()
        _check(_lib.mps_ctx_bytes_allocated(self.handle, ctypes.byref(v)))
        return v.value

    def close(self):
        if self.handle:
            for child in list(self._children):
                child.close()
            _lib.mps_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hamiltonian(_Child):
    _destroy = staticmethod(lambda h: _lib.mps_ham_destroy(h))

    def __init__(self, ctx: Context, ham):
        self._adopt(ctx)
        self.n_qubits = int(ham.n_qubits)
        ops = np.ascontiguousarray(ham.ops, dtype=np.uint8)
        coeffs = np.ascontiguousarray(ham.coeffs, dtype=np.float64)
        self.n_terms = int(ops.shape[0])
        h = ctypes.c_void_p()
        _check(_lib.mps_hamiltonian_create(ctx.handle, self.n_qubits, self.n_terms, _ptr(ops), _ptr(coeffs),
                                           ctypes.byref(h)))
        self.handle = h

    def info(self):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.mps_hamiltonian_info(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"n_terms": a.value, "n_nodes": b.value, "max_level_nodes": c.value}


class Observables(_Child):
    """Rows of complex weights over the strings of a Hamiltonian handle
    (mps_observables_create): row r is sum_e weights[e] <P_{cols[e]}> over
    e in row_ptr[r]:row_ptr[r+1]."""

    _destroy = staticmethod(lambda h: _lib.mps_observables_destroy(h))

    def __init__(self, strings: Hamiltonian, row_ptr, cols, weights):
        self._adopt(strings.ctx)
        self.strings = strings  # the string set must outlive this handle
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        c = np.ascontiguousarray(cols, dtype=np.int32)
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.complex128)).view(np.float64)
        if rp.ndim != 1 or rp.shape[0] < 1:
            raise ValueError("row_ptr needs n_rows + 1 entries")
        self.n_rows = int(rp.shape[0] - 1)
        h = ctypes.c_void_p()
        _check(_lib.mps_observables_create(strings.handle, self.n_rows, _ptr(rp), _ptr(c), _ptr(w),
                                           ctypes.byref(h)))
        self.handle = h


class Circuit(_Child):
    _destroy = staticmethod(lambda h: _lib.mps_circuit_destroy(h))

    def __init__(self, ctx: Context, tmpl):
        self._adopt(ctx)
        self.n_qubits = int(tmpl.n_qubits)
        self.n_params = int(tmpl.n_params)
        self.n_gates = int(tmpl.n_gates)
        arr = template_to_abi(tmpl)
        h = ctypes.c_void_p()
        _check(_lib.mps_circuit_create(ctx.handle, self.n_qubits, _ptr(arr), arr.shape[0], self.n_params,
                                       ctypes.byref(h)))
        self.handle = h


class State(_Child):
    """A right-canonical MPS on the GPU."""

    _destroy = staticmethod(lambda h: _lib.mps_destroy(h))

    def __init__(self, ctx: Context, n_qubits: int, init_bits=None, chi_max: int = 64, precision: str = "fp64",
                 trunc_rel: float = 0.0, svd_fp64: bool = True, svd_max_sweeps: int = 0, svd_tol: float = 0.0,
                 tensor_cores: bool = False):
        self._adopt(ctx)
        self.n = int(n_qubits)
        self.cfg = Config(int(chi_max), PRECISIONS[precision], float(trunc_rel), int(svd_fp64),
                          int(svd_max_sweeps), float(svd_tol), 1 if tensor_cores else 0)
        bits = None if init_bits is None else np.ascontiguousarray(init_bits, dtype=np.uint8)
        h = ctypes.c_void_p()
        _check(_lib.mps_create(ctx.handle, self.n, _ptr(bits), ctypes.byref(self.cfg), ctypes.byref(h)))
        self.handle = h

    def reset(self, init_bits=None):
        bits = None if init_bits is None else np.ascontiguousarray(init_bits, dtype=np.uint8)
        _check(_lib.mps_reset(self.handle, _ptr(bits)))

    def apply_gates(self, gates) -> dict:
        """Apply a GateList; returns the report.  An SVD that reached its sweep
        cap (MPS_ENOTCONV) still updates the state: it is counted in the
        report's ``svd_not_converged`` instead of raising."""
        arr = gates_to_abi(gates)
        rep = Report()
        rc = _lib.mps_apply_gates(self.handle, _ptr(arr), arr.shape[0], ctypes.byref(rep))
        if rc != MPS_ENOTCONV:
            _check(rc)
        return rep.as_dict()

    def apply_circuit(self, circuit: Circuit, theta, device_ptr: int = None):
        """Bind theta (host array, or a device pointer to n_params doubles) and
        apply the circuit; asynchronous on the context stream."""
        if device_ptr is not None:
            _check(_lib.mps_apply_circuit_async(self.handle, circuit.handle, ctypes.c_void_p(int(device_ptr)), 1))
        else:
            th = np.ascontiguousarray(theta, dtype=np.float64)
            if th.shape != (circuit.n_params,):
                raise ValueError(f"theta has shape {th.shape}, circuit takes ({circuit.n_params},)")
            _check(_lib.mps_apply_circuit_async(self.handle, circuit.handle, _ptr(th), 0))

    def energy(self, ham: Hamiltonian, with_norm: bool = False):
        e, nrm = ctypes.c_double(), ctypes.c_double()
        _check(_lib.mps_energy(self.handle, ham.handle, ctypes.byref(e), ctypes.byref(nrm) if with_norm else None))
        return (e.value, nrm.value) if with_norm else e.value

    def energy_async(self, ham: Hamiltonian, device_ptr: int):
        _check(_lib.mps_energy_async(self.handle, ham.handle, ctypes.c_void_p(int(device_ptr))))

    def expectations(self, ham: Hamiltonian) -> np.ndarray:
        out = np.zeros(ham.n_terms)
        _check(_lib.mps_expectations(self.handle, ham.handle, _ptr(out)))
        return out

    def observables(self, obs: Observables) -> np.ndarray:
        """Complex values of every row of ``obs`` for the current state."""
        out = np.zeros(2 * obs.n_rows)
        _check(_lib.mps_observables_eval(self.handle, obs.handle, _ptr(out)))
        return out.view(np.complex128)

    def bond_dims(self) -> np.ndarray:
        out = np.zeros(self.n + 1, dtype=np.int32)
        _check(_lib.mps_bond_dims(self.handle, _ptr(out)))
        return out

    def export(self):
        """(list of B_n arrays (chi_l, 2, chi_r) complex128, list of lam_b arrays)."""
        chi = self.bond_dims()
        nt = int(sum(2 * chi[s] * 2 * chi[s + 1] for s in range(self.n)))
        nl = int(chi.sum())
        t = np.zeros(nt)
        lam = np.zeros(nl)
        _check(_lib.mps_export(self.handle, _ptr(t), nt, _ptr(lam), nl))
        B, L = [], []
        o = 0
        for s in range(self.n):
            cnt = chi[s] * 2 * chi[s + 1]
            z = t[2 * o: 2 * (o + cnt)].view(np.complex128)
            B.append(z.reshape(chi[s], 2, chi[s + 1]).copy())
            o += cnt
        o = 0
        for b in range(self.n + 1):
            L.append(lam[o: o + chi[b]].copy())
            o += chi[b]
        return B, L

    def report(self) -> dict:
        rep = Report()
        _check(_lib.mps_get_report(self.handle, ctypes.byref(rep)))
        return rep.as_dict()


def contract_theta(ctx: Context, precision: str, chi_l: int, chi_m: int, chi_r: int, b_left_ptr: int,
                   b_right_ptr: int, gate, c_out_ptr: int):
    """C = Q (B_q B_{q+1}) on complex64 device arrays (mps_contract_theta);
    asynchronous on the context stream."""
    g = np.ascontiguousarray(np.stack([np.real(gate), np.imag(gate)], axis=-1).reshape(-1), dtype=np.float64)
    if g.shape != (32,):
        raise ValueError("gate must be 4x4")
    _check(_lib.mps_contract_theta(ctx.handle, PRECISIONS[precision], int(chi_l), int(chi_m), int(chi_r),
                                   ctypes.c_void_p(int(b_left_ptr)), ctypes.c_void_p(int(b_right_ptr)), _ptr(g),
                                   ctypes.c_void_p(int(c_out_ptr))))


def truncated_svd(ctx: Context, precision: str, m: int, n: int, c_ptr: int, chi_max: int, trunc_rel: float,
                  svd_fp64: int, s_out_ptr: int, vh_out_ptr: int):
    """Truncated SVD of an m x n device theta (mps_truncated_svd).  Returns
    (k, report, status); MPS_ENOTCONV is returned as the status, with the
    results written, rather than raised."""
    k = ctypes.c_int32()
    rep = Report()
    rc = _lib.mps_truncated_svd(ctx.handle, PRECISIONS[precision], int(m), int(n), ctypes.c_void_p(int(c_ptr)),
                                int(chi_max), float(trunc_rel), int(svd_fp64), ctypes.c_void_p(int(s_out_ptr)),
                                ctypes.c_void_p(int(vh_out_ptr)), ctypes.byref(k), ctypes.byref(rep))
    if rc not in (MPS_OK, MPS_ENOTCONV):
        _check(rc)
    return k.value, rep.as_dict(), rc


def vqe_eval(ctx: Context, requests):
    """requests: list of (State, Circuit, Hamiltonian, theta, init_bits or None).
    Returns (energies, statuses)."""
    n = len(requests)
    reqs = (VqeRequest * n)()
    keep = []
    for i, (st, circ, ham, theta, bits) in enumerate(requests):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        b = None if bits is None else np.ascontiguousarray(bits, dtype=np.uint8)
        keep += [th, b]
        reqs[i] = VqeRequest(st.handle.value, circ.handle.value, ham.handle.value, th.ctypes.data,
                             None if b is None else b.ctypes.data)
    energies = np.zeros(n)
    status = np.zeros(n, dtype=np.int32)
    rc = _lib.vqe_eval(ctx.handle, reqs, n, _ptr(energies), _ptr(status))
    if rc not in (MPS_OK, MPS_ENOTCONV) and np.all((status == MPS_OK) | (status == MPS_ENOTCONV)):
        _check(rc)
    return energies, status


def _requests(requests):
    n = len(requests)
    reqs = (VqeRequest * n)()
    keep = []
    for i, (st, circ, ham, theta, bits) in enumerate(requests):
        if isinstance(theta, int):  # a device pointer
            th_ptr = theta
        else:
            th = np.ascontiguousarray(theta, dtype=np.float64)
            keep.append(th)
            th_ptr = th.ctypes.data
        b = None if bits is None else np.ascontiguousarray(bits, dtype=np.uint8)
        keep.append(b)
        reqs[i] = VqeRequest(st.handle.value, circ.handle.value, ham.handle.value, th_ptr,
                             None if b is None else b.ctypes.data)
    return reqs, keep


def vqe_eval_batch_async(requests, d_energies_ptr: int):
    """Device-resident batch: every theta is a device pointer (int) and the
    energies go to the device array at d_energies_ptr.  Returns the statuses;
    the work is still running on the states' streams."""
    reqs, keep = _requests(requests)
    n = len(requests)
    status = np.zeros(n, dtype=np.int32)
    rc = _lib.vqe_eval_batch_async(reqs, n, ctypes.c_void_p(int(d_energies_ptr)), _ptr(status))
    if rc != MPS_OK:
        _check(rc)
    del keep
    return status


def vqe_eval_batch(requests):
    """Independent evaluations overlapped on the device.  requests: list of
    (State, Circuit, Hamiltonian, theta, init_bits or None) with distinct
    states (each state's context stream carries its work).
    Returns (energies, statuses)."""
    reqs, keep = _requests(requests)
    n = len(requests)
    energies = np.zeros(n)
    status = np.zeros(n, dtype=np.int32)
    rc = _lib.vqe_eval_batch(reqs, n, _ptr(energies), _ptr(status))
    if rc not in (MPS_OK, MPS_ENOTCONV) and np.all((status == MPS_OK) | (status == MPS_ENOTCONV)):
        _check(rc)
    del keep
    return energies, status


class Server:
    """Continuous-batching server of energy evaluations (vqe_submit / vqe_poll)."""

    def __init__(self, device: int = 0, max_slots: int = 8, hbm_budget_bytes: int = 0):
        h = ctypes.c_void_p()
        _check(_lib.mps_server_create(int(device), int(max_slots), int(hbm_budget_bytes), ctypes.byref(h)))
        self.handle = h
        self._keep = []
        _live_servers.add(self)

    def add_fragment(self, circuit: Circuit, ham: Hamiltonian, init_bits=None, chi_max: int = 64,
                     precision: str = "fp32", trunc_rel: float = 1e-5, svd_fp64: bool = False,
                     tensor_cores: bool = False) -> int:
        cfg = Config(int(chi_max), PRECISIONS[precision], float(trunc_rel), int(svd_fp64), 0, 0.0,
                     1 if tensor_cores else 0)
        bits = None if init_bits is None else np.ascontiguousarray(init_bits, dtype=np.uint8)
        out = ctypes.c_int32()
        _check(_lib.mps_server_add_fragment(self.handle, circuit.handle, ham.handle, _ptr(bits), ctypes.byref(cfg),
                                            ctypes.byref(out)))
        self._keep += [circuit, ham]  # must outlive the server
        return out.value

    def submit(self, fragment: int, theta) -> int:
        th = np.ascontiguousarray(theta, dtype=np.float64)
        t = ctypes.c_uint64()
        _check(_lib.vqe_submit(self.handle, int(fragment), _ptr(th), ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1):
        """(energy, latency_ms), or None if not finished within timeout_ms."""
        e, lat = ctypes.c_double(), ctypes.c_double()
        rc = _lib.vqe_poll(self.handle, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(e), ctypes.byref(lat))
        if rc == MPS_ETIMEOUT:
            return None
        if rc != MPS_ENOTCONV:  # the energy of a sweep-cap hit is delivered (see the header)
            _check(rc)
        return e.value, lat.value

    def stats(self) -> dict:
        c, a, q = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        b, pk = ctypes.c_size_t(), ctypes.c_size_t()
        _check(_lib.mps_server_stats(self.handle, ctypes.byref(c), ctypes.byref(a), ctypes.byref(q), ctypes.byref(b),
                                     ctypes.byref(pk)))
        return {"completed": c.value, "active": a.value, "queued": q.value, "bytes": b.value,
                "peak_bytes": pk.value}

    def close(self):
        if self.handle:
            _lib.mps_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
