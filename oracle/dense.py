"""Brute-force dense statevector simulation (oracle pin; small n only).

Qubit 0 is the most significant bit of the amplitude index; a two-qubit gate
on (q, q+1) uses the basis index 2 i_q + i_{q+1}.
"""

import numpy as np

from .mps import PAULI


def basis_state(bits) -> np.ndarray:
    bits = np.asarray(bits, dtype=int)
    n = bits.size
    idx = 0
    for b in bits:
        idx = 2 * idx + int(b)
    psi = np.zeros(1 << n, dtype=complex)
    psi[idx] = 1.0
    return psi


def apply_gate(psi: np.ndarray, n: int, q: int, arity: int, u: np.ndarray) -> np.ndarray:
    if arity == 1:
        t = psi.reshape(1 << q, 2, -1)
        return np.einsum("ij,ajb->aib", u[:2, :2], t).reshape(-1)
    t = psi.reshape(1 << q, 4, -1)
    return np.einsum("ij,ajb->aib", u, t).reshape(-1)


def run(n: int, bits, gates) -> np.ndarray:
    psi = basis_state(np.zeros(n, int) if bits is None else bits)
    for g in range(gates.n_gates):
        psi = apply_gate(psi, n, int(gates.q[g]), int(gates.arity[g]), gates.u[g])
    return psi


def apply_pauli(psi: np.ndarray, ops_row) -> np.ndarray:
    n = len(ops_row)
    t = psi.reshape((2,) * n)
    for j, o in enumerate(ops_row):
        if o:
            t = np.moveaxis(np.tensordot(PAULI[int(o)], t, axes=([1], [j])), 0, j)
    return t.reshape(-1)


def expect_pauli(psi: np.ndarray, ops_row) -> float:
    return float(np.vdot(psi, apply_pauli(psi, ops_row)).real / np.vdot(psi, psi).real)


def energy(psi: np.ndarray, ham) -> float:
    return float(sum(c * expect_pauli(psi, row) for row, c in zip(ham.ops, ham.coeffs)))


def pauli_matrix(ops_row) -> np.ndarray:
    m = np.ones((1, 1), dtype=complex)
    for o in ops_row:
        m = np.kron(m, PAULI[int(o)])
    return m


def hamiltonian_matrix(ham) -> np.ndarray:
    dim = 1 << ham.n_qubits
    H = np.zeros((dim, dim), dtype=complex)
    for row, c in zip(ham.ops, ham.coeffs):
        H += c * pauli_matrix(row)
    return H


def gates_unitary(n: int, gates) -> np.ndarray:
    """Dense unitary of a gate list (columns = images of basis states)."""
    dim = 1 << n
    U = np.eye(dim, dtype=complex)
    for k in range(dim):
        col = U[:, k]
        for g in range(gates.n_gates):
            col = apply_gate(col, n, int(gates.q[g]), int(gates.arity[g]), gates.u[g])
        U[:, k] = col
    return U
