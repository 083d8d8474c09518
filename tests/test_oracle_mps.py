"""Pins of the oracle MPS simulator against the dense statevector, closed forms
and the invariants of the paper's MPS algorithm (CPU only)."""

import numpy as np
import pytest

from oracle import dense as od
from oracle import mps as om
from paper_2303_03681_gb300.inputs import (MASTER_SEED, brickwork_circuit, hf_bits, jw_molecular_hamiltonian,
                                           make_rng, random_integrals, random_local_pauli_sum)


def c1_instance():
    h, g = random_integrals(6, make_rng(MASTER_SEED))
    ham = jw_molecular_hamiltonian(h, g)
    circ = brickwork_circuit(12, 8, make_rng(MASTER_SEED + 1))
    return ham, circ, hf_bits(12, 6)


def test_c1_uncapped_matches_dense_statevector():
    ham, circ, bits = c1_instance()
    assert circ.n_gates == 44
    mps = om.run_circuit(12, bits, circ, chi_max=64, eps_rel=0.0)
    psi = od.run(12, bits, circ)
    fid = abs(np.vdot(psi, om.to_statevector(mps))) ** 2
    assert fid >= 1 - 1e-12
    assert abs(om.energy(mps, ham) - od.energy(psi, ham)) <= 1e-10
    assert mps.bond_dims()[6] == 64


def test_expec2_matches_full_contraction_untruncated():
    ham, circ, bits = c1_instance()
    mps = om.run_circuit(12, bits, circ, chi_max=64)
    sub = range(0, ham.n_terms, 37)
    for k in sub:
        assert abs(om.expect_pauli(mps, ham.ops[k]) - om.expect_pauli_full(mps, ham.ops[k])) <= 1e-12


def test_canonical_form_and_unit_norm():
    _, circ, bits = c1_instance()
    mps = om.run_circuit(12, bits, circ, chi_max=64)
    assert om.canonical_residual(mps) <= 1e-12
    for lam in mps.lam:
        assert abs(np.sum(lam ** 2) - 1.0) <= 1e-12
        assert np.all(np.diff(lam) <= 0)
    assert abs(om.norm_full(mps) - 1.0) <= 1e-12


def test_hastings_identity_after_one_gate():
    """B~_q B~_{q+1} = C (Eq. Bl) and B~_q = U lam~ / lam_{q} (untruncated)."""
    rng = make_rng(5)
    circ = brickwork_circuit(6, 3, rng)
    mps = om.run_circuit(6, None, circ, chi_max=64)
    q = 2
    u4 = brickwork_circuit(2, 1, rng).u[0]
    Bl, Br = mps.B[q], mps.B[q + 1]
    C = np.einsum("ijkl,akld->aijd", u4.reshape(2, 2, 2, 2), np.einsum("aim,mjb->aijb", Bl, Br))
    lam_left = mps.lam[q].copy()
    om.apply_2q(mps, q, u4, chi_max=64)
    C2 = np.einsum("aim,mjb->aijb", mps.B[q], mps.B[q + 1])
    assert np.allclose(C2, C, atol=1e-12)
    # U lam~ = C~ V^dagger; with B~_q = C V^dagger this is lam_{q} B~_q
    Ct = lam_left[:, None, None, None] * C
    Vh = mps.B[q + 1].reshape(mps.B[q + 1].shape[0], -1)
    Ul = Ct.reshape(2 * Bl.shape[0], -1) @ Vh.conj().T
    assert np.allclose(Ul.reshape(mps.B[q].shape), lam_left[:, None, None] * mps.B[q], atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_product_state_single_pauli_values(seed):
    rng = make_rng(seed)
    bits = rng.integers(0, 2, 9)
    mps = om.product_state(bits)
    for j in range(9):
        for op in (1, 2, 3):
            row = np.zeros(9, np.uint8)
            row[j] = op
            want = (1.0 - 2.0 * bits[j]) if op == 3 else 0.0
            assert om.expect_pauli(mps, row) == want
    row = np.zeros(9, np.uint8)
    row[[1, 4, 7]] = 3
    assert om.expect_pauli(mps, row) == np.prod(1.0 - 2.0 * bits[[1, 4, 7]])


def test_single_qubit_gate_is_exact():
    rng = make_rng(3)
    circ = brickwork_circuit(5, 4, rng)
    mps = om.run_circuit(5, None, circ, chi_max=32)
    psi = od.run(5, None, circ)
    u = brickwork_circuit(2, 1, rng).u[0]
    w, _ = np.linalg.qr(u[:2, :2] + 0.3)
    om.apply_1q(mps, 3, w)
    U = np.zeros((4, 4), complex)
    U[:2, :2] = w
    psi = od.apply_gate(psi, 5, 3, 1, U)
    assert abs(abs(np.vdot(psi, om.to_statevector(mps))) - 1) < 1e-12
    assert om.canonical_residual(mps) < 1e-12


def test_truncated_run_invariants():
    n = 14
    circ = brickwork_circuit(n, 10, make_rng(MASTER_SEED + 2))
    exact = om.run_circuit(n, None, circ, chi_max=128)
    trunc = om.run_circuit(n, None, circ, chi_max=12, eps_rel=1e-8)
    assert max(trunc.bond_dims()) == 12
    for lam in trunc.lam:
        assert abs(np.sum(lam ** 2) - 1.0) <= 1e-12
    # B~_{q+1} = V stays exactly right-canonical; B~_q is right-canonical up to
    # the discarded weight of the cut.
    assert om.canonical_residual(trunc) <= 4 * np.sqrt(trunc.stats.discarded_weight) + 1e-10
    f = om.fidelity(exact, trunc)
    assert 0 < trunc.stats.discarded_weight
    assert 1 - f <= 2 * trunc.stats.discarded_weight + 1e-12
    ham = random_local_pauli_sum(n, 40, make_rng(9))
    e_exact = od.energy(od.run(n, None, circ), ham)
    assert abs(om.energy(exact, ham) - e_exact) <= 1e-10


@pytest.mark.parametrize("chi_cap,eps_rel", [(6, 0.0), (64, 0.05)])
def test_single_truncation_is_the_dense_schmidt_truncation(chi_cap, eps_rel):
    """On an exact canonical state the SVD of C~ (Eq. svdtildeC) is the Schmidt
    decomposition across the bond between sites q and q+1, so one truncated
    gate must give the best rank-k approximation of the dense state across
    that cut (Eckart-Young), renormalised: the same state, lam = the k
    largest dense singular values over their norm, and discarded weight
    1 - sum(kept s^2) / sum(s^2).  k follows the truncation rule (chi cap or
    relative threshold)."""
    from paper_2303_03681_gb300.inputs.circuits import haar_su4

    n, q = 10, 4
    rng = make_rng(MASTER_SEED + 20)
    mps = om.run_circuit(n, None, brickwork_circuit(n, 6, rng), chi_max=64)
    u = haar_su4(rng)
    psi = od.apply_gate(om.to_statevector(mps), n, q, 2, u)
    U, s, Vh = np.linalg.svd(psi.reshape(1 << (q + 1), -1), full_matrices=False)
    k = om.truncation_rank(s, chi_cap, eps_rel)
    assert np.count_nonzero(s > 1e-12) > k  # the cut really truncates
    om.apply_2q(mps, q, u, chi_max=chi_cap, eps_rel=eps_rel)
    best = (U[:, :k] * s[:k]) @ Vh[:k]
    best = best.reshape(-1) / np.linalg.norm(s[:k])
    got = om.to_statevector(mps)
    assert mps.B[q].shape[2] == k
    assert abs(abs(np.vdot(best, got)) ** 2 - 1.0) <= 1e-12
    assert np.max(np.abs(mps.lam[q + 1] - s[:k] / np.linalg.norm(s[:k]))) <= 1e-12
    assert abs(mps.stats.discarded_weight - (1 - np.sum(s[:k] ** 2) / np.sum(s ** 2))) <= 1e-12


# -- planted mistakes: each must be caught by the pins above ------------------

def _bad_apply_2q_scaled_c(mps, q, u4, chi_max, eps_rel=0.0, svd=None):
    """Eq. Bl with the lam-scaled C~ in place of C."""
    Bl, Br = mps.B[q], mps.B[q + 1]
    chi_l, chi_r = Bl.shape[0], Br.shape[2]
    C = np.einsum("ijkl,akld->aijd", u4.reshape(2, 2, 2, 2), np.einsum("aim,mjb->aijb", Bl, Br))
    Ct = (mps.lam[q][:, None, None, None] * C).reshape(2 * chi_l, 2 * chi_r)
    _, s, Vh = np.linalg.svd(Ct, full_matrices=False)
    k = om.truncation_rank(s, chi_max, eps_rel)
    nrm = np.linalg.norm(s[:k])
    mps.B[q] = (Ct @ Vh[:k].conj().T / nrm).reshape(chi_l, 2, k)
    mps.B[q + 1] = Vh[:k].reshape(k, 2, chi_r)
    mps.lam[q + 1] = s[:k] / nrm


def test_planted_scaled_c_is_caught(monkeypatch):
    ham, circ, bits = c1_instance()
    monkeypatch.setattr(om, "apply_2q", _bad_apply_2q_scaled_c)
    mps = om.run_circuit(12, bits, circ, chi_max=64)
    psi = od.run(12, bits, circ)
    assert abs(om.energy(mps, ham) - od.energy(psi, ham)) > 1e-6


def test_planted_transposed_gate_is_caught():
    ham, circ, bits = c1_instance()
    bad = type(circ)(circ.n_qubits, circ.q, circ.arity, np.transpose(circ.u, (0, 2, 1)))
    mps = om.run_circuit(12, bits, bad, chi_max=64)
    psi = od.run(12, bits, circ)
    assert abs(om.energy(mps, ham) - od.energy(psi, ham)) > 1e-6


def test_planted_lambda_not_squared_is_caught(monkeypatch):
    ham, circ, bits = c1_instance()
    mps = om.run_circuit(12, bits, circ, chi_max=64)
    good = om.energy(mps, ham)
    orig = om.expect_pauli

    def bad(m, row):
        support = np.nonzero(row)[0]
        if support.size == 0:
            return 1.0
        a, b = support[0], support[-1]
        L = np.diag(m.lam[a]).astype(complex)
        for j in range(a, b + 1):
            L = om._transfer(L, m.B[j], om.PAULI[int(row[j])])
        return float(np.trace(L).real)

    monkeypatch.setattr(om, "expect_pauli", bad)
    assert abs(om.energy(mps, ham) - good) > 1e-6
    monkeypatch.setattr(om, "expect_pauli", orig)
