"""The adaptive Pauli-product ansatz (Methods, "The wave function ansatz for
hydrogen chain simulations") on the CPU.

Pins: the pool equals the Z-stripped, odd-Y Pauli decomposition of the
generalised excitation generators built as dense matrices from ladder
operators; every gradient row equals the dense commutator i[H, P]; the rows
applied to oracle per-string values equal the shift-rule slope of the
energy; the adaptive loop reaches the textbook H2/STO-3G full-CI energy and
respects the variational bound on a random molecule.
"""

import itertools

import numpy as np

from oracle import dense as od
from oracle import fock
from oracle import mps as om
from paper_2303_03681_gb300.adapt import commutator_rows, qubit_adapt
from paper_2303_03681_gb300.inputs import MASTER_SEED, hf_bits, jw_molecular_hamiltonian, make_rng, random_integrals
from paper_2303_03681_gb300.inputs.circuits import gsd_excitations, pauli_product_template, windowed_gsd_pool
from paper_2303_03681_gb300.vqe import sequential_minimize
from test_vqe_loop import DenseEnergy, h2_sto3g, sector_ground_energy


def test_gsd_excitations_by_enumeration():
    orbs = [1, 2, 3]
    so = [2 * p + s for p in orbs for s in (0, 1)]
    got = set(gsd_excitations(orbs))
    singles = {(q, p) for p, q in itertools.permutations(so, 2) if p > q and p % 2 == q % 2}
    doubles = set()
    for a, b, i, j in itertools.product(so, repeat=4):
        if not (a > b and j > i and (a, b) > (j, i)):
            continue
        if sorted([a % 2, b % 2]) != sorted([i % 2, j % 2]):
            continue
        doubles.add((i, j, a, b))
    assert got == singles | doubles
    assert len(got) == len(gsd_excitations(orbs))  # no repeats


def test_pool_structure():
    n_orb = 7
    pool = windowed_gsd_pool(n_orb)
    assert pool.shape[1] == 2 * n_orb
    assert not np.any(pool == 3)
    assert np.all(np.count_nonzero(pool == 2, axis=1) % 2 == 1)
    assert len({r.tobytes() for r in pool}) == pool.shape[0]
    for r in pool:  # the support lies inside one window of 5 orbitals (10 qubits)
        nz = np.nonzero(r)[0]
        assert any(2 * w <= nz[0] and nz[-1] < 2 * w + 10 for w in range(n_orb - 4))


def _pauli_decomposition(M, n):
    out = {}
    for ops in itertools.product(range(4), repeat=n):
        c = np.trace(od.pauli_matrix(ops) @ M) / (1 << n)
        if abs(c) > 1e-12:
            out[tuple(ops)] = c
    return out


def test_pool_is_the_stripped_decomposition_of_the_generators():
    n_orb = 2
    n = 2 * n_orb
    ref = set()
    for exc in gsd_excitations(range(n_orb)):
        G = fock.excitation_generator_matrix(n, exc)
        for ops in _pauli_decomposition(G, n):
            s = tuple(0 if o == 3 else o for o in ops)
            if any(s) and sum(o == 2 for o in s) % 2 == 1:
                ref.add(s)
    assert {tuple(r) for r in windowed_gsd_pool(n_orb)} == ref


def test_rows_are_the_dense_commutators():
    h, g = random_integrals(3, make_rng(MASTER_SEED + 100))
    ham = jw_molecular_hamiltonian(h, g)
    pool = windowed_gsd_pool(3)
    pick = np.concatenate([np.arange(8), np.arange(pool.shape[0] - 8, pool.shape[0])])
    strings, row_ptr, cols, w = commutator_rows(ham, pool[pick])
    H = od.hamiltonian_matrix(ham)
    mats = {}
    for r, j in enumerate(pick):
        P = od.pauli_matrix(pool[j])
        ref = 1j * (H @ P - P @ H)
        got = np.zeros_like(ref)
        for e in range(row_ptr[r], row_ptr[r + 1]):
            c = int(cols[e])
            if c not in mats:
                mats[c] = od.pauli_matrix(strings[c])
            got += w[e] * mats[c]
        assert np.max(np.abs(got - ref)) <= 1e-12
        assert np.max(np.abs(w[row_ptr[r]:row_ptr[r + 1]].imag)) == 0.0


def test_row_gradients_equal_the_shift_rule_slope():
    """Rows applied to oracle (Eq. expec2) per-string values vs
    E(pi/4) - E(-pi/4) for exp(i t P) appended to the circuit."""
    n_orb = 3
    h, g = random_integrals(n_orb, make_rng(MASTER_SEED + 101))
    ham = jw_molecular_hamiltonian(h, g)
    bits = hf_bits(2 * n_orb, 2)
    pool = windowed_gsd_pool(n_orb)
    rng = make_rng(MASTER_SEED + 102)
    chosen = list(rng.choice(pool.shape[0], 4, replace=False))
    theta = rng.uniform(-0.6, 0.6, 4)
    state = om.run_circuit(2 * n_orb, bits, pauli_product_template(2 * n_orb, pool, chosen).bind(theta), 64)
    strings, row_ptr, cols, w = commutator_rows(ham, pool)
    vals = np.array([om.expect_pauli(state, s) for s in strings])
    grad = np.array([(w[row_ptr[j]:row_ptr[j + 1]] @ vals[cols[row_ptr[j]:row_ptr[j + 1]]]).real
                     for j in range(pool.shape[0])])
    shift = []
    for j in range(pool.shape[0]):
        f = DenseEnergy(pauli_product_template(2 * n_orb, pool, chosen + [j]), ham, bits)
        e = f(np.array([np.append(theta, np.pi / 4), np.append(theta, -np.pi / 4)]))
        shift.append(e[0] - e[1])
    assert np.max(np.abs(grad - np.array(shift))) <= 1e-10
    assert np.max(np.abs(grad)) > 1e-2


def dense_gradients(ham, pool, bits):
    strings, row_ptr, cols, w = commutator_rows(ham, pool)

    def grads(tmpl, theta):
        psi = od.run(tmpl.n_qubits, bits, tmpl.bind(theta))
        vals = np.array([od.expect_pauli(psi, s) for s in strings])
        return np.array([(w[row_ptr[j]:row_ptr[j + 1]] @ vals[cols[row_ptr[j]:row_ptr[j + 1]]]).real
                         for j in range(pool.shape[0])])

    return grads


def test_adapt_reaches_h2_full_ci():
    ham = h2_sto3g()
    bits = hf_bits(4, 2)
    pool = windowed_gsd_pool(2)
    res = qubit_adapt(pool, 4, dense_gradients(ham, pool, bits), lambda t: DenseEnergy(t, ham, bits),
                      max_ops=4, grad_tol=1e-7, tol=1e-13)
    assert res.converged and len(res.chosen) <= 3
    assert abs(res.energy - sector_ground_energy(ham, 2)) <= 1e-9


def test_adapt_random_molecule_descends_and_is_variational():
    n_orb, n_e = 4, 4
    h, g = random_integrals(n_orb, make_rng(MASTER_SEED + 103))
    ham = jw_molecular_hamiltonian(h, g)
    bits = hf_bits(2 * n_orb, n_e)
    pool = windowed_gsd_pool(n_orb)
    e_hf = od.energy(od.basis_state(bits), ham)
    res = qubit_adapt(pool, 2 * n_orb, dense_gradients(ham, pool, bits), lambda t: DenseEnergy(t, ham, bits),
                      max_ops=5, grad_tol=1e-8, optimizer=sequential_minimize, max_sweeps=6, tol=1e-9)
    assert len(res.energies) == 5
    assert res.energies[0] < e_hf - 1e-3
    assert np.all(np.diff(res.energies) <= 1e-10)
    assert res.energy >= sector_ground_energy(ham, n_e) - 1e-10


def test_commuting_pool_strings_give_empty_rows_and_adapt_stops():
    ham = h2_sto3g()
    pool = np.array([[0, 0, 0, 0], [3, 3, 0, 0], [2, 1, 1, 1]], np.uint8)  # I and ZZ commute with every Z/I term
    strings, row_ptr, cols, w = commutator_rows(ham, pool)
    assert row_ptr[1] == row_ptr[0] and row_ptr.size == 4 and row_ptr[-1] == cols.size
    res = qubit_adapt(pool, 4, lambda t, th: np.zeros(pool.shape[0]), lambda t: None, max_ops=3, grad_tol=1e-6)
    assert res.converged and res.chosen == [] and res.energy is None and res.max_gradients == [0.0]


def test_symplectic_products_on_several_words():
    """Packed-word phases and products against a per-site table on 70- and
    130-qubit strings (two and three 64-bit words)."""
    from paper_2303_03681_gb300.adapt import _pauli_product_phase
    from paper_2303_03681_gb300.inputs.hamiltonian import ops_to_symplectic, symplectic_to_ops

    # sigma_a sigma_b = i^E[a, b] sigma_{a xor b} for I, X, Y, Z = 0, 1, 2, 3
    E = np.array([[0, 0, 0, 0], [0, 0, 1, 3], [0, 3, 0, 1], [0, 1, 3, 0]])
    rng = make_rng(MASTER_SEED + 104)
    for n in (70, 130):
        A = rng.integers(0, 4, (300, n)).astype(np.uint8)
        B = rng.integers(0, 4, n).astype(np.uint8)
        ax, az = ops_to_symplectic(A)
        bx, bz = ops_to_symplectic(B[None])
        assert np.array_equal(symplectic_to_ops(ax, az, n), A)
        e = _pauli_product_phase(ax, az, bx[0], bz[0])
        assert np.array_equal(e, E[A, B[None, :]].sum(axis=1) % 4)
        assert np.array_equal(symplectic_to_ops(ax ^ bx[0], az ^ bz[0], n), A ^ B[None, :])


def test_pool_chunks_cover_the_pool_within_the_cap():
    from paper_2303_03681_gb300.adapt import pool_chunks

    h, g = random_integrals(4, make_rng(MASTER_SEED + 105))
    ham = jw_molecular_hamiltonian(h, g)
    pool = windowed_gsd_pool(4)
    _, row_ptr, _, _ = commutator_rows(ham, pool)
    sizes = np.diff(row_ptr)
    cap = int(sizes.max() * 5)
    chunks = pool_chunks(ham, pool, cap)
    assert chunks[0][0] == 0 and chunks[-1][1] == pool.shape[0]
    assert all(a[1] == b[0] for a, b in zip(chunks, chunks[1:]))
    assert all(sizes[lo:hi].sum() <= cap for lo, hi in chunks) and len(chunks) > 1
    # per-chunk rows equal the slices of the whole-pool rows
    for lo, hi in chunks:
        s2, rp2, c2, w2 = commutator_rows(ham, pool[lo:hi])
        assert np.array_equal(np.diff(rp2), sizes[lo:hi])
