"""Right-canonical MPS simulator in FP64 (oracle; test infrastructure only).

Follows the paper's Methods, subsection "MPS algorithm for quantum circuit
simulation" and "The implementation of UCCSD with matrix product states":

* Eq. (mps): c_{i1..iN} = B^{i1} B^{i2} ... B^{iN}; site tensor ``B[n]`` has
  shape (chi_{n-1}, 2, chi_n) and index order [alpha_{n-1}, i_n, alpha_n].
* Eq. (rightcanonicalcondition): sum_{i, alpha_n} B B^* = identity.
* bond singular values: ``lam[b]`` sits on the bond left of site b
  (lam[0] = lam[N] = [1]); a gate on sites (q, q+1) reads lam[q] and
  replaces lam[q+1].
* one-qubit gate: B~^{i} = sum_{i'} Q_{i i'} B^{i'}.
* two-qubit gate (Hastings): C = Q . (B_q B_{q+1}); C~ = lam_{q} C
  (Eq. tildeC); SVD(C~) = U lam~ V (Eq. svdtildeC) with truncation;
  B~_q = C V^dagger (Eq. Bl, unscaled C); B~_{q+1} = V; lam_{q+1} = lam~.
* expectation values: Eq. (expec1) / (expec2) - lam^2 on the bond left of
  the first non-identity site, transfer products up to the last one, the
  right side is the identity by right-canonicity.

Readings where the paper is silent (stated once, used throughout):

* truncation keeps k = min(chi_max, #{s_i > eps_rel * s_1}) >= 1 singular
  values (eps_rel = 0 keeps every nonzero one);
* the kept part is renormalised: lam = s[:k] / ||s[:k]|| and
  B~_q = C V_k^dagger / ||s[:k]||, so the state keeps unit norm;
* the identity string has expectation sum(lam[0]^2) = 1.
"""

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

from . import svd_jacobi

PAULI = {
    0: np.eye(2, dtype=complex),
    1: np.array([[0, 1], [1, 0]], dtype=complex),
    2: np.array([[0, -1j], [1j, 0]], dtype=complex),
    3: np.array([[1, 0], [0, -1]], dtype=complex),
}


@dataclass
class TruncationStats:
    discarded_weight: float = 0.0  # sum over gates of 1 - sum(kept s^2) / sum(s^2)
    max_chi: int = 1
    degenerate_cuts: int = 0  # cuts at chi_max inside a (near-)degenerate pair
    min_kept_sv: float = 1.0


@dataclass
class MPS:
    B: list
    lam: list
    stats: TruncationStats = field(default_factory=TruncationStats)

    @property
    def n(self) -> int:
        return len(self.B)

    def bond_dims(self):
        return [b.shape[0] for b in self.B] + [self.B[-1].shape[2]]

    def copy(self) -> "MPS":
        return MPS([b.copy() for b in self.B], [l.copy() for l in self.lam],
                   TruncationStats(**vars(self.stats)))


def product_state(bits) -> MPS:
    """chi = 1 MPS of the computational basis state |bits> (Hartree-Fock or |0..0>)."""
    bits = np.asarray(bits, dtype=int)
    B = []
    for b in bits:
        t = np.zeros((1, 2, 1), dtype=complex)
        t[0, int(b), 0] = 1.0
        B.append(t)
    lam = [np.ones(1) for _ in range(len(bits) + 1)]
    return MPS(B, lam)


def apply_1q(mps: MPS, q: int, u2: np.ndarray) -> None:
    """One-qubit gate on site q (Methods, single-qubit gate equation)."""
    mps.B[q] = np.einsum("ij,ajb->aib", u2, mps.B[q])


def truncation_rank(s: np.ndarray, chi_max: int, eps_rel: float) -> int:
    """Number of singular values kept (reading of 'truncate the small singular
    values below a certain threshold or simply reserve the largest few')."""
    if eps_rel > 0.0:
        k = int(np.count_nonzero(s > eps_rel * s[0]))
    else:
        k = int(np.count_nonzero(s > 0.0))
    return max(1, min(k, int(chi_max)))


def svd_robust(A: np.ndarray):
    """SVD of Eq. svdtildeC, A = U diag(s) Vh with s descending.

    LAPACK's divide-and-conquer driver (zgesdd) is tried first.  It can stop
    with "SVD did not converge" on some inputs (seen on an aarch64 OpenBLAS
    build), so the QR-iteration driver (zgesvd) is tried next, and the
    one-sided Jacobi SVD of Algorithm 1 (``svd_jacobi``) last.  All three
    compute the same decomposition; only the rounding differs."""
    try:
        return np.linalg.svd(A, full_matrices=False)
    except np.linalg.LinAlgError:
        pass
    try:
        return scipy.linalg.svd(A, full_matrices=False, lapack_driver="gesvd")
    except (np.linalg.LinAlgError, ValueError):
        pass
    return svd_jacobi.one_sided_jacobi_svd(A)


def apply_2q(mps: MPS, q: int, u4: np.ndarray, chi_max: int, eps_rel: float = 0.0,
             svd=None) -> None:
    """Two-qubit gate on sites (q, q+1) with the Hastings update (Methods,
    Eqs. tildeC, svdtildeC and Bl).  ``svd`` defaults to ``svd_robust``
    (LAPACK zgesdd, with zgesvd and Algorithm 1 as fallbacks)."""
    Bl, Br = mps.B[q], mps.B[q + 1]
    chi_l, chi_r = Bl.shape[0], Br.shape[2]
    theta = np.einsum("aim,mjb->aijb", Bl, Br)
    Q = u4.reshape(2, 2, 2, 2)  # Q[i, j, i', j']
    C = np.einsum("ijkl,akld->aijd", Q, theta)
    Cmat = C.reshape(2 * chi_l, 2 * chi_r)
    Ct = mps.lam[q][:, None] * C.reshape(chi_l, 4 * chi_r)
    Ct = Ct.reshape(2 * chi_l, 2 * chi_r)
    if svd is None:
        _, s, Vh = svd_robust(Ct)
    else:
        _, s, Vh = svd(Ct)
    k = truncation_rank(s, chi_max, eps_rel)
    total = float(np.sum(s * s))
    kept = float(np.sum(s[:k] * s[:k]))
    nrm = np.sqrt(kept)
    Vk = Vh[:k]
    mps.B[q] = (Cmat @ Vk.conj().T / nrm).reshape(chi_l, 2, k)
    mps.B[q + 1] = Vk.reshape(k, 2, chi_r)
    mps.lam[q + 1] = s[:k] / nrm
    st = mps.stats
    st.discarded_weight += (1.0 - kept / total) if total > 0 else 0.0
    st.max_chi = max(st.max_chi, k)
    st.min_kept_sv = min(st.min_kept_sv, float(s[k - 1] / nrm))
    if k < s.size and k == chi_max and s[k] > 0 and abs(s[k - 1] - s[k]) <= 1e-10 * s[k - 1]:
        st.degenerate_cuts += 1


def apply_gates(mps: MPS, gates, chi_max: int, eps_rel: float = 0.0, svd=None) -> MPS:
    """Apply a GateList in order."""
    for g in range(gates.n_gates):
        q = int(gates.q[g])
        if int(gates.arity[g]) == 1:
            apply_1q(mps, q, gates.u[g][:2, :2])
        else:
            apply_2q(mps, q, gates.u[g], chi_max, eps_rel, svd)
    return mps


def _transfer(L: np.ndarray, B: np.ndarray, P: np.ndarray) -> np.ndarray:
    """L'[b, d] = sum conj(B[a, i, b]) L[a, c] P[i, j] B[c, j, d]."""
    return np.einsum("aib,ac,ij,cjd->bd", B.conj(), L, P, B, optimize=True)


def expect_pauli(mps: MPS, ops_row) -> float:
    """<P> by Eq. (expec1)/(expec2): lam^2 on the bond left of the first
    non-identity site m, transfers over sites m..n, trace at the right end."""
    ops_row = np.asarray(ops_row)
    support = np.nonzero(ops_row)[0]
    if support.size == 0:
        return float(np.sum(mps.lam[0] ** 2))
    m, n = int(support[0]), int(support[-1])
    L = np.diag(mps.lam[m] ** 2).astype(complex)
    for j in range(m, n + 1):
        L = _transfer(L, mps.B[j], PAULI[int(ops_row[j])])
    return float(np.trace(L).real)


def energy(mps: MPS, ham) -> float:
    """E = sum_k c_k <P_k>, each string evaluated on its own (no prefix sharing)."""
    return float(sum(c * expect_pauli(mps, row) for row, c in zip(ham.ops, ham.coeffs)))


def expect_pauli_full(mps: MPS, ops_row) -> float:
    """<psi|P|psi> / <psi|psi> by transfer contraction over all sites from the
    left boundary; uses no canonical form."""
    L = np.ones((1, 1), dtype=complex)
    N = np.ones((1, 1), dtype=complex)
    for j in range(mps.n):
        L = _transfer(L, mps.B[j], PAULI[int(ops_row[j])])
        N = _transfer(N, mps.B[j], PAULI[0])
    return float((L[0, 0] / N[0, 0]).real)


def norm_full(mps: MPS) -> float:
    N = np.ones((1, 1), dtype=complex)
    for j in range(mps.n):
        N = _transfer(N, mps.B[j], PAULI[0])
    return float(N[0, 0].real)


def energy_full(mps: MPS, ham) -> float:
    return float(sum(c * expect_pauli_full(mps, row) for row, c in zip(ham.ops, ham.coeffs)))


def canonical_residual(mps: MPS) -> float:
    """max_n || sum_{i} B^i B^{i dagger} - I ||_F (Eq. rightcanonicalcondition)."""
    worst = 0.0
    for B in mps.B:
        chi_l = B.shape[0]
        M = B.reshape(chi_l, -1)
        worst = max(worst, float(np.linalg.norm(M @ M.conj().T - np.eye(chi_l))))
    return worst


def to_statevector(mps: MPS) -> np.ndarray:
    """Dense amplitudes, qubit 0 the most significant bit (small n only)."""
    psi = mps.B[0].reshape(2, -1)
    for B in mps.B[1:]:
        psi = (psi @ B.reshape(B.shape[0], -1)).reshape(-1, B.shape[2])
    return psi.reshape(-1)


def fidelity(a: MPS, b: MPS) -> float:
    """|<a|b>|^2 / (<a|a><b|b>) by transfer contraction."""
    L = np.ones((1, 1), dtype=complex)
    for Ba, Bb in zip(a.B, b.B):
        L = np.einsum("aib,ac,cid->bd", Ba.conj(), L, Bb, optimize=True)
    ab = L[0, 0]
    return float(abs(ab) ** 2 / (norm_full(a) * norm_full(b)))


def run_circuit(n_qubits: int, init_bits, gates, chi_max: int, eps_rel: float = 0.0) -> MPS:
    bits = np.zeros(n_qubits, dtype=int) if init_bits is None else init_bits
    return apply_gates(product_state(bits), gates, chi_max, eps_rel)


def vqe_energy(template, theta, init_bits, ham, chi_max: int, eps_rel: float = 0.0) -> float:
    """One energy evaluation: reset to the reference state, apply the circuit
    bound to theta, evaluate E."""
    mps = run_circuit(template.n_qubits, init_bits, template.bind(theta), chi_max, eps_rel)
    return energy(mps, ham)
