"""Reduced density matrices of a statevector, by their definition (oracle;
test infrastructure only).

The paper's DMET subsection (Methods, "The DMET method") evaluates the
fragment energy and electron count from the 1-RDM <a+_p a_q> and the 2-RDM
<a+_p a+_q a_r a_s>.  Here both are computed on a dense statevector by
applying the ladder operators to occupation bit strings (``fock``), with no
Pauli strings involved:

* gamma[P, Q] = <psi| a+_P a_Q |psi>                (spin orbitals)
* Gamma[P, Q, R, S] = <psi| a+_P a+_Q a_R a_S |psi>  (spin orbitals)
* spin-summed, chemists' order:
  D[p, q] = sum_s gamma[ps, qs],
  d[p, q, r, s] = sum_{s1, s2} Gamma[p s1, r s2, s s2, q s1],
  so that E = sum h_pq D_pq + 1/2 sum (pq|rs) d_pqrs for the Hamiltonian of
  the "Unitary coupled cluster" subsection, and N = trace(D).
Interleaved spin orbitals (qubit 2p + s), qubit 0 the most significant bit.
"""

import numpy as np

from .fock import apply_monomial


def one_rdm(psi: np.ndarray, n_so: int) -> np.ndarray:
    psi = psi / np.linalg.norm(psi)
    g = np.zeros((n_so, n_so), dtype=complex)
    for P in range(n_so):
        for Q in range(n_so):
            g[P, Q] = np.vdot(psi, apply_monomial(psi, n_so, [(P, True), (Q, False)], 1.0))
    return g


def two_rdm(psi: np.ndarray, n_so: int) -> np.ndarray:
    psi = psi / np.linalg.norm(psi)
    G = np.zeros((n_so,) * 4, dtype=complex)
    for P in range(n_so):
        for Q in range(n_so):
            if P == Q:
                continue
            for R in range(n_so):
                for S in range(n_so):
                    if R == S:
                        continue
                    G[P, Q, R, S] = np.vdot(psi, apply_monomial(psi, n_so, [(P, True), (Q, True), (R, False),
                                                                          (S, False)], 1.0))
    return G


def spatial_rdms(gamma: np.ndarray, Gamma: np.ndarray):
    """Spin-summed D (n_orb, n_orb) and chemists'-order d (n_orb,)*4."""
    n = gamma.shape[0] // 2
    D = np.zeros((n, n), dtype=complex)
    d = np.zeros((n,) * 4, dtype=complex)
    for s in (0, 1):
        D += gamma[s::2, s::2]
    for s1 in (0, 1):
        for s2 in (0, 1):
            # d[p, q, r, s] += Gamma[p s1, r s2, s s2, q s1]
            d += np.transpose(Gamma[s1::2, s2::2, s2::2, s1::2], (0, 3, 1, 2))
    return D, d


def rdm_energy(h: np.ndarray, g: np.ndarray, D: np.ndarray, d: np.ndarray) -> float:
    return float(np.real(np.sum(h * D) + 0.5 * np.sum(g * d)))
