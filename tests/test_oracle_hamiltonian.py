"""Pins of the Hamiltonian generator and of the oracle's energy routes (CPU).

* The JW Pauli sum equals the second-quantised Hamiltonian built on
  occupation bit strings (independent code) on random vectors.
* The chi = 1 Hartree-Fock MPS energy equals the closed-form determinant
  energy (paper: the UCC reference state |Phi_0> is the HF determinant).
* The textbook H2/STO-3G integrals reproduce the printed HF and FCI energies,
  and minimising the oracle's UCCSD-MPS energy over theta reaches the FCI
  energy (the paper reports UCCSD-MPS is exact for STO-3G H2).
"""

import json
import os

import numpy as np
import pytest

from oracle import dense as od
from oracle import fock as of
from oracle import mps as om
from paper_2303_03681_gb300.inputs import (MASTER_SEED, hf_bits, jw_molecular_hamiltonian, make_rng,
                                           random_integrals, random_local_pauli_sum, uccsd_template)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("n_orb", [2, 3, 4, 6])
def test_jw_sum_matches_occupation_basis(n_orb):
    rng = make_rng(MASTER_SEED + 100 + n_orb)
    h, g = random_integrals(n_orb, rng)
    ham = jw_molecular_hamiltonian(h, g)
    dim = 1 << (2 * n_orb)
    for _ in range(2):
        v = rng.normal(size=dim) + 1j * rng.normal(size=dim)
        ref = of.molecular_hamiltonian_action(h, g, v)
        got = sum(c * od.apply_pauli(v, row) for row, c in zip(ham.ops, ham.coeffs))
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_integral_symmetry():
    h, g = random_integrals(5, make_rng(MASTER_SEED))
    assert np.array_equal(h, h.T)
    for perm in ["qprs", "pqsr", "rspq", "qpsr", "srqp", "rsqp", "srpq"]:
        assert np.array_equal(g, np.einsum("pqrs->" + perm, g))


@pytest.mark.parametrize("n_orb,n_e", [(2, 2), (4, 4), (6, 6), (6, 4), (8, 6)])
def test_hf_product_state_energy_matches_closed_form(n_orb, n_e):
    rng = make_rng(MASTER_SEED + 7 * n_orb + n_e)
    h, g = random_integrals(n_orb, rng)
    ham = jw_molecular_hamiltonian(h, g)
    mps = om.product_state(hf_bits(2 * n_orb, n_e))
    e_closed = of.hf_energy(h, g, n_e)
    assert abs(om.energy(mps, ham) - e_closed) <= 1e-12 * max(1.0, abs(e_closed))


def test_c1_term_count_and_hermiticity():
    h, g = random_integrals(6, make_rng(MASTER_SEED))
    ham = jw_molecular_hamiltonian(h, g)
    assert ham.n_qubits == 12
    assert ham.n_terms == len({r.tobytes() for r in ham.ops})  # distinct strings
    H = od.hamiltonian_matrix(jw_molecular_hamiltonian(*random_integrals(3, make_rng(1))))
    assert np.allclose(H, H.conj().T, atol=1e-13)


def _h2():
    with open(os.path.join(GOLDEN, "h2_sto3g.json")) as f:
        d = json.load(f)
    h = np.array(d["h"])
    g = np.zeros((2, 2, 2, 2))
    g[0, 0, 0, 0] = d["J11"]
    g[1, 1, 1, 1] = d["J22"]
    g[0, 0, 1, 1] = g[1, 1, 0, 0] = d["J12"]
    for idx in [(0, 1, 0, 1), (1, 0, 1, 0), (0, 1, 1, 0), (1, 0, 0, 1)]:
        g[idx] = d["K12"]
    return d, h, g


def test_h2_textbook_hf_and_fci():
    d, h, g = _h2()
    ham = jw_molecular_hamiltonian(h, g)
    e_hf = om.energy(om.product_state(hf_bits(4, 2)), ham)
    assert abs(e_hf - d["printed_hf_electronic_energy"]) < 2e-4
    # 2x2 CI between |1a 1b> and |2a 2b> (closed form), printed FCI energy
    h11 = 2 * h[0, 0] + d["J11"]
    h22 = 2 * h[1, 1] + d["J22"]
    e_ci = 0.5 * (h11 + h22) - np.sqrt(0.25 * (h11 - h22) ** 2 + d["K12"] ** 2)
    assert abs(e_ci - d["printed_fci_electronic_energy"]) < 2e-4
    w = np.linalg.eigvalsh(od.hamiltonian_matrix(ham))
    assert abs(w[0] - e_ci) < 1e-12


def test_h2_uccsd_mps_vqe_reaches_fci():
    from scipy.optimize import minimize

    d, h, g = _h2()
    ham = jw_molecular_hamiltonian(h, g)
    tmpl = uccsd_template(4, 2)
    bits = hf_bits(4, 2)
    w = np.linalg.eigvalsh(od.hamiltonian_matrix(ham))
    res = minimize(lambda th: om.vqe_energy(tmpl, th, bits, ham, chi_max=4), np.zeros(tmpl.n_params),
                   method="BFGS", options={"gtol": 1e-10})
    assert abs(res.fun - w[0]) < 1e-9


def test_local_pauli_sum_pool():
    ham = random_local_pauli_sum(20, 100, make_rng(MASTER_SEED))
    assert ham.n_terms == 100
    assert len({r.tobytes() for r in ham.ops}) == 100
    for row in ham.ops:
        nz = np.nonzero(row)[0]
        assert 1 <= nz.size <= 2 and nz[-1] - nz[0] <= 2
