"""Pins of the circuit generators (CPU): Haar SU(4), brickwork layout, and the
compiled UCCSD Pauli exponentials against scipy.linalg.expm of each
excitation generator built from dense JW ladder matrices."""

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import dense as od
from oracle import fock as of
from paper_2303_03681_gb300.inputs import (brickwork_circuit, haar_su4, make_rng, pauli_exponential_template,
                                           uccsd_excitations, uccsd_template)
from paper_2303_03681_gb300.inputs.circuits import excitation_generator_paulis


def test_haar_su4_is_special_unitary():
    rng = make_rng(0)
    for _ in range(20):
        u = haar_su4(rng)
        assert np.allclose(u @ u.conj().T, np.eye(4), atol=1e-13)
        assert abs(np.linalg.det(u) - 1) < 1e-12


def test_brickwork_layout():
    c = brickwork_circuit(12, 8, make_rng(1))
    assert c.n_gates == 4 * 6 + 4 * 5
    assert list(c.q[:6]) == [0, 2, 4, 6, 8, 10]
    assert list(c.q[6:11]) == [1, 3, 5, 7, 9]


def test_excitation_counts():
    assert len(uccsd_excitations(50, 10)) == 200 + 13800
    assert len(uccsd_excitations(4, 2)) == 3


@pytest.mark.parametrize("n_so,n_e", [(6, 2), (8, 4)])
def test_each_generator_compiles_to_expm(n_so, n_e):
    rng = make_rng(n_so)
    for exc in uccsd_excitations(n_so, n_e):
        ops, c = excitation_generator_paulis(n_so, exc)
        G = of.excitation_generator_matrix(n_so, exc)
        # tau - tau^dagger = sum_k i c_k P_k
        S = sum(1j * ck * od.pauli_matrix(row) for row, ck in zip(ops, c))
        assert np.allclose(S, G, atol=1e-13)
        theta = rng.uniform(-1, 1)
        tmpl = pauli_exponential_template(n_so, [(row, 0, ck) for row, ck in zip(ops, c)], 1)
        U = od.gates_unitary(n_so, tmpl.bind([theta]))
        assert np.allclose(U, expm(theta * G), atol=1e-12)


def test_uccsd_circuit_is_the_trotter_product():
    n_so, n_e = 6, 2
    rng = make_rng(17)
    tmpl = uccsd_template(n_so, n_e)
    theta = rng.uniform(-0.05, 0.05, tmpl.n_params)
    U = od.gates_unitary(n_so, tmpl.bind(theta))
    ref = np.eye(1 << n_so, dtype=complex)
    for k, exc in enumerate(uccsd_excitations(n_so, n_e)):
        ref = expm(theta[k] * of.excitation_generator_matrix(n_so, exc)) @ ref
    assert np.allclose(U, ref, atol=1e-12)


def test_gate_count_formula():
    tmpl = uccsd_template(10, 4)
    total = 0
    for exc in uccsd_excitations(10, 4):
        ops, _ = excitation_generator_paulis(10, exc)
        for row in ops:
            nz = np.nonzero(row)[0]
            total += 2 * (nz[-1] - nz[0]) - 1
    assert tmpl.n_two_qubit == total
    assert np.all(tmpl.arity == 2)
    assert np.count_nonzero(tmpl.param >= 0) == tmpl.meta["n_pauli_exponentials"]
