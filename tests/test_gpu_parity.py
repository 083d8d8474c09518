"""GPU parity: the CUDA path (through the C-ABI) against the FP64 CPU oracle.

Tolerances:
* complex128 states (MPS_PREC_FP64): |dE| <= 1e-10 Ha, fidelity >= 1 - 1e-12,
  singular values within 1e-10 - the two sides differ only in rounding order
  (LAPACK zgesdd vs the GPU one-sided Jacobi);
* complex64 states (MPS_PREC_FP32, FP64 SVD): |dE| <= 1e-6 Ha and fidelity
  >= 1 - 1e-8, the accuracy bar of the method's mixed-precision form.
Truncated runs compare at equal chi_max and eps_rel and check that no cut
fell inside a degenerate pair (where the truncated state is not unique).
"""

import numpy as np
import pytest

from gpu_helpers import spectra_close, to_oracle
from oracle import dense as od
from oracle import mps as om
from paper_2303_03681_gb300.inputs import (MASTER_SEED, CircuitTemplate, brickwork_circuit, hf_bits,
                                           jw_molecular_hamiltonian, make_rng, random_integrals,
                                           random_local_pauli_sum, uccsd_template)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mps():
    from paper_2303_03681_gb300 import mps as m

    return m


@pytest.fixture(scope="module")
def ctx(mps):
    return mps.Context(0)


def c1():
    h, g = random_integrals(6, make_rng(MASTER_SEED))
    return jw_molecular_hamiltonian(h, g), brickwork_circuit(12, 8, make_rng(MASTER_SEED + 1)), hf_bits(12, 6)


@pytest.fixture(scope="module")
def c1_ref():
    ham, circ, bits = c1()
    ref = om.run_circuit(12, bits, circ, chi_max=64)
    return ham, circ, bits, ref, om.energy(ref, ham)


def test_c1_fp64_matches_oracle_and_dense(mps, ctx, c1_ref):
    ham, circ, bits, ref, e_ref = c1_ref
    st = mps.State(ctx, 12, bits, chi_max=64, precision="fp64")
    rep = st.apply_gates(circ)
    H = mps.Hamiltonian(ctx, ham)
    e, nrm = st.energy(H, with_norm=True)
    assert abs(e - e_ref) <= 1e-10
    assert abs(e - od.energy(od.run(12, bits, circ), ham)) <= 1e-10
    assert abs(nrm - 1.0) <= 1e-12
    assert list(st.bond_dims()) == ref.bond_dims()
    got = to_oracle(st)
    assert spectra_close(got.lam, ref.lam, 1e-10)
    assert om.fidelity(got, ref) >= 1 - 1e-12
    assert om.canonical_residual(got) <= 1e-10
    assert rep["two_qubit_gates"] == 44 and rep["svd_not_converged"] == 0


def test_c1_per_term_expectations(mps, ctx, c1_ref):
    """The trie energy against Eq. expec2 evaluated string by string on the same state."""
    ham, circ, bits, _, _ = c1_ref
    st = mps.State(ctx, 12, bits, chi_max=64, precision="fp64")
    st.apply_gates(circ)
    vals = st.expectations(mps.Hamiltonian(ctx, ham))
    got = to_oracle(st)
    want = np.array([om.expect_pauli(got, row) for row in ham.ops])
    assert np.max(np.abs(vals - want)) <= 1e-12


def test_c1_fp32_storage(mps, ctx, c1_ref):
    ham, circ, bits, ref, e_ref = c1_ref
    st = mps.State(ctx, 12, bits, chi_max=64, precision="fp32", svd_fp64=True)
    st.apply_gates(circ)
    e = st.energy(mps.Hamiltonian(ctx, ham))
    assert abs(e - e_ref) <= 1e-6
    assert om.fidelity(to_oracle(st), ref) >= 1 - 1e-8


@pytest.mark.parametrize("precision,svd64", [("fp64", True), ("fp32", True), ("fp32", False)])
def test_truncated_brickwork_ragged_chi(mps, ctx, precision, svd64):
    n, chi = 16, 24  # chi spans two 16-wide tiles with a ragged tail; SVD 48 x 48
    circ = brickwork_circuit(n, 12, make_rng(MASTER_SEED + 3))
    ham = random_local_pauli_sum(n, 200, make_rng(MASTER_SEED + 4))
    ref = om.run_circuit(n, None, circ, chi_max=chi, eps_rel=1e-10)
    assert ref.stats.degenerate_cuts == 0
    st = mps.State(ctx, n, None, chi_max=chi, precision=precision, trunc_rel=1e-10, svd_fp64=svd64)
    rep = st.apply_gates(circ)
    assert rep["degenerate_cuts"] == 0
    assert list(st.bond_dims()) == ref.bond_dims()
    e = st.energy(mps.Hamiltonian(ctx, ham))
    tol_e, tol_f = (1e-9, 1e-11) if precision == "fp64" else (1e-5, 1e-6)
    if not svd64:
        tol_e, tol_f = 1e-4, 1e-5
    assert abs(e - om.energy(ref, ham)) <= tol_e
    assert om.fidelity(to_oracle(st), ref) >= 1 - tol_f
    assert abs(rep["discarded_weight"] - ref.stats.discarded_weight) <= max(1e-9, 1e-3 * ref.stats.discarded_weight)


def test_svd_global_memory_path(mps, ctx):
    """theta of 192 x 192 complex128 does not fit in shared memory: the Jacobi
    SVD runs on global memory."""
    n, chi = 14, 96
    circ = brickwork_circuit(n, 9, make_rng(MASTER_SEED + 5))
    ref = om.run_circuit(n, None, circ, chi_max=chi, eps_rel=1e-12)
    st = mps.State(ctx, n, None, chi_max=chi, precision="fp64", trunc_rel=1e-12)
    st.apply_gates(circ)
    got = to_oracle(st)
    assert list(st.bond_dims()) == ref.bond_dims()
    assert max(ref.bond_dims()) == 96
    assert spectra_close(got.lam, ref.lam, 1e-9)
    assert om.fidelity(got, ref) >= 1 - 1e-10


@pytest.mark.parametrize("n,layers,precision,svd64,chi", [(14, 10, "fp32", False, 128), (14, 10, "fp32", False, 60),
                                                          (13, 9, "fp32", True, 64), (16, 14, "fp64", True, 100),
                                                          (16, 14, "fp64", True, 128), (18, 12, "fp32", True, 256),
                                                          (14, 10, "fp32", True, 128), (14, 10, "fp32", 2, 128)])
def test_cluster_svd_path(mps, ctx, n, layers, precision, svd64, chi):
    """Thetas with 2 chi_r >= 96 columns take the thread-block-cluster Jacobi
    (8 CTAs below 192 columns, 16 above); ragged chi pads the column blocks.
    FP64 at chi 128 and chi 256 have stacked columns too long for shared
    memory at the capacity: they live in global memory, and in shared memory
    again for the gates whose actual bond dimensions fit.  Complex64 states
    with svd_fp64 = 1 take the mixed FP32-then-FP64 sweeps, svd_fp64 = 2 the
    all-FP64 ones.

    Complex64 runs compare where truncation does not decide the outcome
    (chi_max at the exact rank, or a chi = 60 cap on a shallow circuit whose
    spectrum has a gap there): heavily truncated random circuits amplify any
    rounding difference, so an FP32 run and the FP64 oracle follow different
    truncated states there."""
    circ = brickwork_circuit(n, layers, make_rng(MASTER_SEED + 12))
    trunc = 1e-5 if precision == "fp32" else 1e-12
    ref = om.run_circuit(n, None, circ, chi_max=chi, eps_rel=trunc)
    st = mps.State(ctx, n, None, chi_max=chi, precision=precision, trunc_rel=trunc, svd_fp64=svd64)
    rep = st.apply_gates(circ)
    assert rep["svd_not_converged"] == 0
    got = to_oracle(st)
    ham = random_local_pauli_sum(n, 200, make_rng(MASTER_SEED + 13))
    e = st.energy(mps.Hamiltonian(ctx, ham))
    dw = max(rep["discarded_weight"], ref.stats.discarded_weight)
    print(f"\ncluster n={n} chi={chi} {precision} svd64={svd64}: dE={e - om.energy(ref, ham):.3e} "
          f"1-F={1 - om.fidelity(got, ref):.3e} dw={dw:.3e} chi={max(st.bond_dims())}/{max(ref.bond_dims())}")
    if precision == "fp64":
        assert list(st.bond_dims()) == ref.bond_dims()
        assert spectra_close(got.lam, ref.lam, 1e-9)
        assert abs(e - om.energy(ref, ham)) <= 1e-9
        assert om.fidelity(got, ref) >= 1 - 1e-10
    else:
        # FP64-accurate SVD (svd_fp64 1: FP32 sweeps then FP64 ones; 2: all FP64)
        # leaves only the complex64 storage rounding
        f = om.fidelity(got, ref)
        assert 1 - f <= (1e-9 if svd64 else 1e-6) + 4 * dw
        # two unit states a, b with |<a|b>|^2 = F differ by ||a - b|| <= sqrt(2 (1 - F)) (up to a phase), so
        # |<a|H|a> - <b|H|b>| <= 2 ||H|| ||a - b|| with ||H|| <= sum |c_k|; plus the complex64 storage rounding
        bound = 2 * float(np.sum(np.abs(ham.coeffs))) * np.sqrt(2 * max(1 - f, 0.0))
        assert abs(e - om.energy(ref, ham)) <= 1e-5 + bound
        # truncation leaves B~_q right-canonical only up to the discarded weight,
        # on both sides alike
        assert om.canonical_residual(got) <= om.canonical_residual(ref) + 1e-3


def test_uccsd_template_through_vqe_eval(mps, ctx):
    n_so, n_e = 8, 4
    rng = make_rng(MASTER_SEED + 6)
    h, g = random_integrals(n_so // 2, rng)
    ham = jw_molecular_hamiltonian(h, g)
    tmpl = uccsd_template(n_so, n_e)
    bits = hf_bits(n_so, n_e)
    circ = mps.Circuit(ctx, tmpl)
    H = mps.Hamiltonian(ctx, ham)
    st = mps.State(ctx, n_so, bits, chi_max=32, precision="fp64")
    thetas = [rng.uniform(-0.5, 0.5, tmpl.n_params) for _ in range(3)]
    energies, status = mps.vqe_eval(ctx, [(st, circ, H, th, bits) for th in thetas])
    assert list(status) == [0, 0, 0]
    for th, e in zip(thetas, energies):
        e_ref = om.vqe_energy(tmpl, th, bits, ham, chi_max=32)
        e_dense = od.energy(od.run(n_so, bits, tmpl.bind(th)), ham)
        assert abs(e - e_ref) <= 1e-10
        assert abs(e - e_dense) <= 1e-10
    again, _ = mps.vqe_eval(ctx, [(st, circ, H, thetas[0], bits)])
    assert again[0] == energies[0]  # deterministic


def test_one_qubit_gates_and_mixed_lists(mps, ctx):
    n = 7
    rng = make_rng(8)
    base = brickwork_circuit(n, 5, rng)
    q, ar, u = list(base.q), list(base.arity), list(base.u)
    for k in range(10):
        x = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
        w, _ = np.linalg.qr(x)
        m = np.zeros((4, 4), complex)
        m[:2, :2] = w
        pos = int(rng.integers(0, len(q)))
        q.insert(pos, int(rng.integers(0, n)))
        ar.insert(pos, 1)
        u.insert(pos, m)
    gl = type(base)(n, np.array(q, np.int32), np.array(ar, np.int32), np.array(u))
    ham = random_local_pauli_sum(n, 40, make_rng(9))
    st = mps.State(ctx, n, None, chi_max=16, precision="fp64")
    st.apply_gates(gl)
    psi = od.run(n, None, gl)
    assert abs(st.energy(mps.Hamiltonian(ctx, ham)) - od.energy(psi, ham)) <= 1e-10


def test_edge_cases(mps, ctx):
    # two qubits, chi_max = 1 (product-state truncation), identity terms, last-site terms
    circ = brickwork_circuit(2, 3, make_rng(10))
    ops = np.array([[0, 0], [0, 3], [3, 0], [1, 2], [0, 1]], np.uint8)
    coeffs = np.array([0.5, 1.0, -2.0, 0.25, 0.75])
    from paper_2303_03681_gb300.inputs import PauliSum

    ham = PauliSum(2, ops, coeffs)
    for chi in (1, 2):
        st = mps.State(ctx, 2, [1, 0], chi_max=chi, precision="fp64")
        st.apply_gates(circ)
        ref = om.run_circuit(2, [1, 0], circ, chi_max=chi)
        assert abs(st.energy(mps.Hamiltonian(ctx, ham)) - om.energy(ref, ham)) <= 1e-12
    # empty gate list and an identity-only Hamiltonian
    st = mps.State(ctx, 5, [1, 1, 0, 1, 0], chi_max=4)
    st.apply_gates(brickwork_circuit(5, 0, make_rng(0)))
    assert st.energy(mps.Hamiltonian(ctx, PauliSum(5, np.zeros((1, 5), np.uint8), np.array([3.25])))) == 3.25
    z = np.zeros((5, 5), np.uint8)
    np.fill_diagonal(z, 3)
    vals = st.expectations(mps.Hamiltonian(ctx, PauliSum(5, z, np.ones(5))))
    assert list(vals) == [-1.0, -1.0, 1.0, -1.0, 1.0]
    assert st.energy(mps.Hamiltonian(ctx, PauliSum(5, np.zeros((0, 5), np.uint8), np.zeros(0)))) == 0.0


def test_invalid_inputs_raise(mps, ctx):
    st = mps.State(ctx, 4, None, chi_max=4)
    bad = brickwork_circuit(4, 1, make_rng(0))
    bad.q[0] = 3  # (3, 4) is outside a 4-qubit chain
    with pytest.raises(mps.MpsError) as ei:
        st.apply_gates(bad)
    assert ei.value.status == mps.MPS_EINVAL
    with pytest.raises(mps.MpsError):
        st.reset([0, 2, 0, 0])
    from paper_2303_03681_gb300.inputs import PauliSum

    with pytest.raises(mps.MpsError):
        mps.Hamiltonian(ctx, PauliSum(4, np.full((1, 4), 7, np.uint8), np.ones(1)))
    with pytest.raises(mps.MpsError):
        st.energy(mps.Hamiltonian(ctx, PauliSum(5, np.zeros((1, 5), np.uint8), np.ones(1))))
    with pytest.raises(mps.MpsError):
        mps.State(ctx, 4, None, chi_max=0)
    # the state is still usable after rejected calls
    st.apply_gates(brickwork_circuit(4, 2, make_rng(1)))
    assert st.bond_dims()[2] >= 1


def test_allocation_cap_gives_enomem(mps):
    c = mps.Context(0)
    c.set_alloc_limit(1 << 16)
    with pytest.raises(mps.MpsError) as ei:
        mps.State(c, 40, None, chi_max=256)
    assert ei.value.status == mps.MPS_ENOMEM
    assert c.bytes_allocated() == 0
    c.set_alloc_limit(0)
    st = mps.State(c, 6, None, chi_max=4)
    assert st.bond_dims().sum() == 7


def test_batch_results_equal_single_results(mps):
    """Each evaluation gives the same energy alone (vqe_eval) and in a batch of
    concurrent evaluations on separate streams (vqe_eval_batch)."""
    n_so, n_e = 8, 4
    rng = make_rng(MASTER_SEED + 31)
    h, g = random_integrals(n_so // 2, rng)
    ham = jw_molecular_hamiltonian(h, g)
    tmpl = uccsd_template(n_so, n_e)
    bits = hf_bits(n_so, n_e)
    thetas = [rng.uniform(-0.3, 0.3, tmpl.n_params) for _ in range(4)]
    ctxs = [mps.Context(0) for _ in thetas]
    circ = mps.Circuit(ctxs[0], tmpl)
    H = mps.Hamiltonian(ctxs[0], ham)
    states = [mps.State(c, n_so, bits, chi_max=16, precision="fp64") for c in ctxs]
    batch, status = mps.vqe_eval_batch([(s, circ, H, th, bits) for s, th in zip(states, thetas)])
    assert list(status) == [0] * len(thetas)
    for s, c, th, e in zip(states, ctxs, thetas, batch):
        alone, st2 = mps.vqe_eval(c, [(s, circ, H, th, bits)])
        assert st2[0] == 0 and alone[0] == e
        assert abs(e - om.vqe_energy(tmpl, th, bits, ham, chi_max=16)) <= 1e-10
    _, status = mps.vqe_eval_batch([(states[0], circ, H, thetas[0], bits), (states[0], circ, H, thetas[1], bits)])
    assert list(status) == [mps.MPS_OK, mps.MPS_EINVAL]  # a state may serve one request of a batch
