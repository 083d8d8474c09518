"""Occupation-number-basis checks of the Hamiltonian and the ansatz (oracle).

These build the second-quantised operators of the paper's "Unitary coupled
cluster" subsection directly on occupation bit strings (or as dense JW
matrices from the definition a_j = Z^{(x)j} (x) |0><1| (x) I), sharing no
code with the Pauli-string generator they check.
"""

import numpy as np


def _apply_ladder(states, signs, valid, n, j, dagger):
    bit = np.int64(1) << np.int64(n - 1 - j)
    occ = (states & bit) != 0
    ok = valid & (~occ if dagger else occ)
    above = states >> np.int64(n - j)  # occupation bits of sites 0..j-1
    parity = np.zeros_like(states)
    x = above.copy()
    while np.any(x):
        parity ^= x & 1
        x >>= 1
    new_states = states ^ bit
    new_signs = np.where(parity & 1, -signs, signs)
    return np.where(ok, new_states, states), np.where(ok, new_signs, signs), ok


def apply_monomial(vec, n, ops, weight):
    """weight * prod(ops) |vec>, ops = [(site, dagger), ...] left to right."""
    dim = 1 << n
    states = np.arange(dim, dtype=np.int64)
    signs = np.ones(dim)
    valid = np.ones(dim, dtype=bool)
    for site, dag in reversed(ops):
        states, signs, valid = _apply_ladder(states, signs, valid, n, site, dag)
    out = np.zeros_like(vec)
    np.add.at(out, states[valid], weight * signs[valid] * vec[valid])
    return out


def molecular_hamiltonian_action(h, g, vec):
    """H |vec> with H = sum h_pq a+_ps a_qs + 1/2 sum (pq|rs) a+_ps a+_rt a_st a_qs
    (interleaved spin orbitals, qubit 0 the most significant bit)."""
    n_orb = h.shape[0]
    n = 2 * n_orb
    out = np.zeros_like(vec)
    for p in range(n_orb):
        for q in range(n_orb):
            for s in (0, 1):
                if h[p, q] != 0.0:
                    out += apply_monomial(vec, n, [(2 * p + s, True), (2 * q + s, False)], h[p, q])
    for p in range(n_orb):
        for q in range(n_orb):
            for r in range(n_orb):
                for s_ in range(n_orb):
                    v = 0.5 * g[p, q, r, s_]
                    if v == 0.0:
                        continue
                    for a in (0, 1):
                        for b in (0, 1):
                            P, Q, R, S = 2 * p + a, 2 * q + a, 2 * r + b, 2 * s_ + b
                            if P == R or Q == S:
                                continue
                            out += apply_monomial(vec, n, [(P, True), (R, True), (S, False), (Q, False)], v)
    return out


def hf_energy(h, g, n_electrons: int) -> float:
    """Closed-shell determinant energy in chemists' notation:
    E = 2 sum_i h_ii + sum_ij [2 (ii|jj) - (ij|ji)], i, j over occupied orbitals."""
    occ = range(n_electrons // 2)
    e = 2.0 * sum(h[i, i] for i in occ)
    e += sum(2.0 * g[i, i, j, j] - g[i, j, j, i] for i in occ for j in occ)
    return float(e)


def ladder_matrix(n: int, j: int, dagger: bool) -> np.ndarray:
    """Dense JW ladder operator on n qubits, built from its definition."""
    Z = np.diag([1.0, -1.0]).astype(complex)
    lower = np.array([[0, 1], [0, 0]], dtype=complex)
    m = np.ones((1, 1), dtype=complex)
    for k in range(n):
        m = np.kron(m, Z if k < j else (lower if k == j else np.eye(2)))
    return m.conj().T if dagger else m


def excitation_generator_matrix(n: int, exc) -> np.ndarray:
    """Dense tau - tau^dagger for a single (i, a) or double (i, j, a, b)."""
    if len(exc) == 2:
        i, a = exc
        tau = ladder_matrix(n, a, True) @ ladder_matrix(n, i, False)
    else:
        i, j, a, b = exc
        tau = (ladder_matrix(n, a, True) @ ladder_matrix(n, b, True)
               @ ladder_matrix(n, j, False) @ ladder_matrix(n, i, False))
    return tau - tau.conj().T
