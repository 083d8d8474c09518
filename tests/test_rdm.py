"""Reduced density matrices (Methods, "The DMET method") on the CPU.

Pins of the oracle (oracle/rdm.py, ladder operators on occupation bit
strings): the Hartree-Fock closed form, Hermiticity, occupation numbers in
[0, 1], trace = N, the partial trace sum_Q Gamma[P, Q, Q, S] = (N - 1)
gamma[P, S], antisymmetry, and the energy identity
E = sum h D + 1/2 sum (pq|rs) d against the Pauli-sum energy.

Host logic of the GPU path (paper_2303_03681_gb300/rdm.py): every row's
Pauli combination equals the dense Jordan-Wigner product of ladder matrices
built from their definition, and the rows applied to oracle per-string
expectation values reproduce the oracle RDMs (real UCCSD states and complex
brickwork states).
"""

import numpy as np
import pytest

from oracle import dense as od
from oracle import fock
from oracle import mps as om
from oracle import rdm as orr
from paper_2303_03681_gb300.inputs import (MASTER_SEED, brickwork_circuit, hf_bits, jw_molecular_hamiltonian,
                                           make_rng, random_integrals, uccsd_template)
from paper_2303_03681_gb300.rdm import KINDS, merged_rows, rdm_rows


def uccsd_state(n_orb, n_e, seed):
    rng = make_rng(MASTER_SEED + seed)
    h, g = random_integrals(n_orb, rng)
    tmpl = uccsd_template(2 * n_orb, n_e)
    theta = rng.uniform(-0.4, 0.4, tmpl.n_params)
    bits = hf_bits(2 * n_orb, n_e)
    return h, g, jw_molecular_hamiltonian(h, g), tmpl.bind(theta), bits


def definition_matrix(n_so, kind, idx):
    L = lambda j, dag: fock.ladder_matrix(n_so, j, dag)  # noqa: E731
    if kind == "1rdm":
        P, Q = idx
        return L(P, True) @ L(Q, False)
    if kind == "2rdm":
        P, Q, R, S = idx
        return L(P, True) @ L(Q, True) @ L(R, False) @ L(S, False)
    if kind == "D":
        p, q = idx
        return sum(L(2 * p + s, True) @ L(2 * q + s, False) for s in (0, 1))
    p, q, r, s = idx
    return sum(L(2 * p + a, True) @ L(2 * r + b, True) @ L(2 * s + b, False) @ L(2 * q + a, False)
               for a in (0, 1) for b in (0, 1))


@pytest.mark.parametrize("n_so,kind", [(4, "1rdm"), (4, "2rdm"), (4, "D"), (4, "d"), (6, "1rdm"), (6, "D")])
def test_rows_are_the_jordan_wigner_products(n_so, kind):
    strings, row_ptr, cols, w, shape = rdm_rows(n_so, kind)
    mats = [od.pauli_matrix(s) for s in strings]
    for r, idx in enumerate(np.ndindex(*shape)):
        got = sum((w[e] * mats[cols[e]] for e in range(row_ptr[r], row_ptr[r + 1])),
                  np.zeros((1 << n_so,) * 2, complex))
        assert np.max(np.abs(got - definition_matrix(n_so, kind, idx))) <= 1e-14, (kind, idx)


def test_hartree_fock_closed_form():
    n_so, n_e = 6, 2
    occ = hf_bits(n_so, n_e).astype(float)
    psi = od.basis_state(hf_bits(n_so, n_e))
    g1 = orr.one_rdm(psi, n_so)
    g2 = orr.two_rdm(psi, n_so)
    assert np.max(np.abs(g1 - np.diag(occ))) == 0.0
    d = np.eye(n_so)
    ref = (np.einsum("p,q,ps,qr->pqrs", occ, occ, d, d) - np.einsum("p,q,pr,qs->pqrs", occ, occ, d, d))
    assert np.max(np.abs(g2 - ref)) == 0.0


def test_oracle_rdm_invariants_and_energy_identity():
    n_orb, n_e = 4, 4
    h, g, ham, gates, bits = uccsd_state(n_orb, n_e, 90)
    psi = od.run(2 * n_orb, bits, gates)
    n_so = 2 * n_orb
    g1 = orr.one_rdm(psi, n_so)
    g2 = orr.two_rdm(psi, n_so)
    assert np.max(np.abs(g1 - g1.conj().T)) <= 1e-14
    occ = np.linalg.eigvalsh(g1)
    assert occ.min() >= -1e-12 and occ.max() <= 1 + 1e-12
    assert abs(np.trace(g1) - n_e) <= 1e-12
    assert np.max(np.abs(np.einsum("pqqs->ps", g2) - (n_e - 1) * g1)) <= 1e-12
    assert np.max(np.abs(g2 + np.transpose(g2, (1, 0, 2, 3)))) <= 1e-14
    assert np.max(np.abs(g2 + np.transpose(g2, (0, 1, 3, 2)))) <= 1e-14
    D, d = orr.spatial_rdms(g1, g2)
    assert abs(np.trace(D) - n_e) <= 1e-12
    assert abs(orr.rdm_energy(h, g, D, d) - od.energy(psi, ham)) <= 1e-11


@pytest.mark.parametrize("state", ["uccsd", "brickwork"])
def test_rows_on_oracle_string_values_give_the_oracle_rdms(state):
    """The GPU path with its kernels replaced by the oracle: per-string
    values from Eq. expec2 on the oracle MPS, then the row sums."""
    if state == "uccsd":
        _, _, _, gates, bits = uccsd_state(3, 2, 91)
        n_so = 6
    else:
        n_so, bits = 6, None
        gates = brickwork_circuit(n_so, 5, make_rng(MASTER_SEED + 92))
    mps = om.run_circuit(n_so, bits, gates, chi_max=64)
    psi = om.to_statevector(mps)
    strings, row_ptr, cols, w, layout = merged_rows(n_so, KINDS)
    vals = np.array([om.expect_pauli(mps, s) for s in strings])
    rows = np.array([w[row_ptr[r]:row_ptr[r + 1]] @ vals[cols[row_ptr[r]:row_ptr[r + 1]]]
                     for r in range(row_ptr.size - 1)])
    out = {k: rows[off: off + int(np.prod(shape))].reshape(shape) for k, off, shape in layout}
    g1, g2 = orr.one_rdm(psi, n_so), orr.two_rdm(psi, n_so)
    D, d = orr.spatial_rdms(g1, g2)
    for k, ref in (("1rdm", g1), ("2rdm", g2), ("D", D), ("d", d)):
        assert np.max(np.abs(out[k] - ref)) <= 1e-12, k
    if state == "brickwork":
        assert np.max(np.abs(g1.imag)) > 1e-3  # complex RDMs: the imaginary weights matter


def test_row_builder_arguments_and_layout():
    with pytest.raises(ValueError):
        rdm_rows(5, "1rdm")
    with pytest.raises(ValueError):
        rdm_rows(4, "3rdm")
    strings, row_ptr, cols, w, layout = merged_rows(4, ("1rdm", "D"))
    assert [(k, off, shape) for k, off, shape in layout] == [("1rdm", 0, (4, 4)), ("D", 16, (2, 2))]
    assert row_ptr.size == 16 + 4 + 1 and row_ptr[0] == 0 and np.all(np.diff(row_ptr) >= 0)
    assert cols.min() >= 0 and cols.max() < strings.shape[0] and row_ptr[-1] == cols.size == w.size
    assert len({s.tobytes() for s in strings}) == strings.shape[0]
    # vanishing monomials (a+_P a+_P) give empty rows
    _, rp2, _, _, _ = rdm_rows(4, "2rdm")
    assert rp2[1] - rp2[0] == 0  # Gamma[0, 0, 0, 0]
