"""Adaptive Pauli-product ansatz for long fragments (Methods, "The wave
function ansatz for hydrogen chain simulations").

The paper's hydrogen-chain circuits are products of exp(i theta_j P_j) over
strings of a pool (``inputs.windowed_gsd_pool``: generalised singles and
doubles within 5 consecutive orbitals, Z-stripped, odd-Y strings), grown in
the manner of qubit-ADAPT-VQE (Tang et al., PRX Quantum 2, 020310 (2021)):
at the current state |psi>, append the pool string with the largest energy
gradient and re-optimise all angles.

Appending exp(i t P) to the circuit gives E(t) = <psi|e^{-itP} H e^{itP}|psi>,
whose slope at t = 0 is g_P = <psi| i[H, P] |psi>.  With H = sum_k c_k P_k,
i[P_k, P] = 2 i P_k P when the two strings anticommute (0 otherwise), and
P_k P = i^e Q with e odd, so

    g_P = sum_{k: P_k anticommutes with P} -2 i^(e_k - 1) c_k <Q_k>,

real weights over the product strings Q_k.  Every pool gradient is therefore
one row over a common set of strings, and one energy-kernel pass over that set
plus one row-sum launch (``mps_observables_eval``) gives all of them at
once.  ``commutator_rows`` builds the rows; ``ObservableGradients`` evaluates
them on the GPU; ``qubit_adapt`` runs the loop with any gradient and energy
providers (the optimisers of ``vqe``).
"""

from dataclasses import dataclass, field

import numpy as np

from .inputs.circuits import pauli_product_template
from .inputs.hamiltonian import PauliSum, _popcount, ops_to_symplectic, symplectic_to_ops
from .vqe import sequential_minimize

def _pauli_product_phase(x1, z1, x2, z2):
    """For strings P_1 = (x1, z1) (packed words, (T, W)) and P_2 = (x2, z2)
    ((W,)), the exponent e (mod 4) of P_1 P_2 = i^e Q: each site contributes
    +1 for the cyclic pairs XY, YZ, ZX (XY = iZ, ...) and -1 for YX, ZY, XZ."""
    X1, Y1, Z1 = x1 & ~z1, x1 & z1, ~x1 & z1
    X2, Y2, Z2 = x2 & ~z2, x2 & z2, ~x2 & z2
    cyc = _popcount((X1 & Y2) | (Y1 & Z2) | (Z1 & X2))
    anti = _popcount((Y1 & X2) | (Z1 & Y2) | (X1 & Z2))
    return (cyc - anti) % 4


def commutator_rows(ham, pool: np.ndarray):
    """Rows g_j = <i[H, pool_j]> over the product strings.

    The strings are handled as packed (x, z) bit words, so one pool string
    costs a few word operations per Hamiltonian term.  Returns (strings
    (T, n) uint8, row_ptr (len(pool) + 1,), cols int32, weights complex
    (real values))."""
    ops = np.asarray(ham.ops, dtype=np.uint8)
    c = np.asarray(ham.coeffs, dtype=float)
    n = ops.shape[1]
    pool = np.asarray(pool, dtype=np.uint8).reshape(-1, n)
    hx, hz = ops_to_symplectic(ops)
    px, pz = ops_to_symplectic(pool)
    keys, rows_j, w = [], [], []
    for j in range(pool.shape[0]):
        e = _pauli_product_phase(hx, hz, px[j], pz[j])
        anti = (e % 2) == 1  # odd exponent: the two strings anticommute
        if not anti.any():
            continue
        keys.append(np.concatenate([hx[anti] ^ px[j], hz[anti] ^ pz[j]], axis=1))
        rows_j.append(np.full(int(anti.sum()), j, np.int64))
        w.append(np.where(e[anti] == 1, -2.0, 2.0) * c[anti])
    W = hx.shape[1]
    if not keys:
        return np.zeros((0, n), np.uint8), np.zeros(pool.shape[0] + 1, np.int64), np.zeros(0, np.int32), \
            np.zeros(0, complex)
    Q = np.ascontiguousarray(np.concatenate(keys))
    rj = np.concatenate(rows_j)
    ww = np.concatenate(w)
    void = Q.view(np.dtype((np.void, Q.dtype.itemsize * Q.shape[1]))).ravel()
    _, first, inv = np.unique(void, return_index=True, return_inverse=True)
    inv = inv.reshape(-1)
    strings = symplectic_to_ops(Q[first, :W], Q[first, W:], n)
    order = np.lexsort((inv, rj))  # by row, then column
    rj, cols, ww = rj[order], inv[order], ww[order]
    row_ptr = np.searchsorted(rj, np.arange(pool.shape[0] + 1)).astype(np.int64)
    return strings.astype(np.uint8), row_ptr, cols.astype(np.int32), ww.astype(complex)


def pool_chunks(ham, pool: np.ndarray, max_entries: int):
    """Split the pool into consecutive chunks whose commutator rows hold at
    most ``max_entries`` entries each (a string anticommuting with k terms
    of H adds k entries; a single string may exceed the cap on its own)."""
    hx, hz = ops_to_symplectic(np.asarray(ham.ops, dtype=np.uint8))
    px, pz = ops_to_symplectic(np.asarray(pool, dtype=np.uint8))
    counts = [int(np.count_nonzero(_pauli_product_phase(hx, hz, px[j], pz[j]) % 2)) for j in range(px.shape[0])]
    chunks, lo, acc = [], 0, 0
    for j, k in enumerate(counts):
        if j > lo and acc + k > max_entries:
            chunks.append((lo, j))
            lo, acc = j, 0
        acc += k
    if lo < len(counts):
        chunks.append((lo, len(counts)))
    return chunks


@dataclass
class AdaptResult:
    chosen: list  # pool indices, in circuit order
    theta: np.ndarray
    energy: float  # measured energy of the final circuit; None if no string was added
    converged: bool  # largest pool gradient fell below grad_tol
    energies: list = field(default_factory=list)  # energy after each growth step
    max_gradients: list = field(default_factory=list)


def qubit_adapt(pool: np.ndarray, n_qubits: int, gradients, energy_factory, max_ops: int = 20,
                grad_tol: float = 1e-4, optimizer=sequential_minimize, **opt_kwargs) -> AdaptResult:
    """Grow prod_k exp(i theta_k P_{chosen_k}) one pool string at a time.

    ``gradients(template, theta) -> (len(pool),)`` gives the slope of the
    energy for appending each pool string at the state template(theta);
    ``energy_factory(template) -> energy_batch`` gives an evaluator for the
    optimiser.  New angles start at 0; every step re-optimises all angles."""
    chosen, theta = [], np.zeros(0)
    energies, gmax = [], []
    energy = None
    converged = False
    for _ in range(max_ops):
        tmpl = pauli_product_template(n_qubits, pool, chosen)
        g = np.asarray(gradients(tmpl, theta), dtype=float)
        j = int(np.argmax(np.abs(g)))
        gmax.append(float(abs(g[j])))
        if abs(g[j]) < grad_tol:
            converged = True
            break
        chosen.append(j)
        theta = np.append(theta, 0.0)
        tmpl = pauli_product_template(n_qubits, pool, chosen)
        res = optimizer(energy_factory(tmpl), theta, **opt_kwargs)
        theta, energy = res.theta, res.energy
        energies.append(energy)
    return AdaptResult(chosen, theta, energy, converged, energies, gmax)


class ObservableGradients:
    """All pool gradients on the GPU: for each chunk of the pool
    (``pool_chunks``, at most ``max_entries`` row entries), the product
    strings of ``commutator_rows`` as one string set and the rows as one
    Observables handle; a state is reset to ``init_bits`` and given the
    current circuit on every call, then every chunk is evaluated on it."""

    def __init__(self, ctx, ham, pool, init_bits=None, max_entries: int = 1 << 24, **state_kwargs):
        from . import mps

        self._mps = mps
        self.ctx = ctx
        self.n_qubits = int(ham.n_qubits)
        self.n_pool = int(np.asarray(pool).shape[0])
        self.bits = None if init_bits is None else np.ascontiguousarray(init_bits, dtype=np.uint8)
        self.chunks = []
        for lo, hi in pool_chunks(ham, pool, max_entries):
            strings, row_ptr, cols, weights = commutator_rows(ham, np.asarray(pool)[lo:hi])
            h = mps.Hamiltonian(ctx, PauliSum(self.n_qubits, strings, np.ones(strings.shape[0])))
            self.chunks.append((lo, hi, h, mps.Observables(h, row_ptr, cols, weights)))
        self.state = mps.State(ctx, self.n_qubits, self.bits, **state_kwargs)

    def __call__(self, template, theta) -> np.ndarray:
        mps = self._mps
        self.state.reset(self.bits)
        circ = None
        if template.n_gates:
            circ = mps.Circuit(self.ctx, template)
            self.state.apply_circuit(circ, np.asarray(theta, dtype=float))
        # observables() synchronises the stream, so the circuit is released
        # only after its gates have run
        g = np.zeros(self.n_pool)
        for lo, hi, _, obs in self.chunks:
            g[lo:hi] = self.state.observables(obs).real
        return g
