"""GPU parity of the tensor-core environment contractions (complex64 states,
tcgen05 TF32 with the hi/lo split, FP32 accumulation).

Each string's expectation value from the GPU is compared with the oracle's
Eq. expec2 contraction of the same exported state, so the only difference is
the rounding of the environment contractions.  The tensor-core path must be
within an absolute 1e-6 per string (the energy bar of the method's accuracy
target) and no less accurate than the FP32 CUDA-core path (at most 3x its
largest error, or 2e-7); its energy must equal
sum_k c_k <P_k> of its own values.  Sizes cover one and several 128-row tiles,
ragged tiles (chi = 100, 200) and the bond dimensions 1 and 2 at the edges.
"""

import numpy as np
import pytest

from gpu_helpers import to_oracle
from oracle import mps as om
from paper_2303_03681_gb300.inputs import (MASTER_SEED, brickwork_circuit, hf_bits, jw_molecular_hamiltonian,
                                           make_rng, random_integrals, random_local_pauli_sum, uccsd_template)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mps():
    from paper_2303_03681_gb300 import mps as m

    return m


@pytest.fixture(scope="module")
def ctx(mps):
    return mps.Context(0)


def _errors(mps, ctx, st, ham, idx=None):
    H = mps.Hamiltonian(ctx, ham)
    vals = st.expectations(H)
    e = st.energy(H)
    assert abs(e - float(np.dot(ham.coeffs, vals))) <= 1e-9 * max(1.0, float(np.sum(np.abs(ham.coeffs))))
    got = to_oracle(st)
    idx = np.arange(ham.n_terms) if idx is None else idx
    want = np.array([om.expect_pauli(got, ham.ops[k]) for k in idx])
    return float(np.max(np.abs(vals[idx] - want))), e


def _pair(mps, ctx, n, bits, gates, chi, trunc=0.0):
    out = []
    for tc in (False, True):
        st = mps.State(ctx, n, bits, chi_max=chi, precision="fp32", trunc_rel=trunc, svd_fp64=True, tensor_cores=tc)
        st.apply_gates(gates)
        out.append(st)
    return out


def test_c1_tensor_cores_match_oracle(mps, ctx):
    h, g = random_integrals(6, make_rng(MASTER_SEED))
    ham = jw_molecular_hamiltonian(h, g)
    circ = brickwork_circuit(12, 8, make_rng(MASTER_SEED + 1))
    simt, tc = _pair(mps, ctx, 12, hf_bits(12, 6), circ, 64)
    err_simt, e_simt = _errors(mps, ctx, simt, ham)
    err_tc, e_tc = _errors(mps, ctx, tc, ham)
    assert err_tc <= 1e-6 and err_tc <= max(3 * err_simt, 2e-7), (err_tc, err_simt)
    assert abs(e_tc - e_simt) <= 1e-4


@pytest.mark.parametrize("n,layers,chi,trunc", [(14, 10, 100, 0.0), (18, 12, 200, 0.0), (16, 10, 256, 1e-5)])
def test_tiles_and_ragged_edges(mps, ctx, n, layers, chi, trunc):
    rng = make_rng(MASTER_SEED + 300 + n)
    circ = brickwork_circuit(n, layers, rng)
    ham = random_local_pauli_sum(n, 80, make_rng(MASTER_SEED + 301 + n))
    simt, tc = _pair(mps, ctx, n, None, circ, chi, trunc)
    assert max(tc.bond_dims()) > 64  # several column tiles at least
    err_simt, _ = _errors(mps, ctx, simt, ham)
    err_tc, _ = _errors(mps, ctx, tc, ham)
    assert err_tc <= 1e-6 and err_tc <= max(3 * err_simt, 2e-7), (err_tc, err_simt)


def test_product_state_and_two_sites(mps, ctx):
    """chi = 1 everywhere (K = 1, a single ragged tile) and the smallest chain."""
    ham = random_local_pauli_sum(6, 40, make_rng(MASTER_SEED + 310))
    st = mps.State(ctx, 6, np.array([1, 0, 1, 1, 0, 0], np.uint8), chi_max=8, precision="fp32", tensor_cores=True)
    err, _ = _errors(mps, ctx, st, ham)
    assert err <= 1e-6
    ham2 = random_local_pauli_sum(2, 15, make_rng(MASTER_SEED + 311))
    st2 = mps.State(ctx, 2, None, chi_max=4, precision="fp32", tensor_cores=True)
    st2.apply_gates(brickwork_circuit(2, 3, make_rng(MASTER_SEED + 312)))
    err2, _ = _errors(mps, ctx, st2, ham2)
    assert err2 <= 1e-6


def test_c2_prefix_tensor_cores(mps, ctx):
    """50 qubits, chi_max = 128, the 571,876-string Hamiltonian: sampled strings
    against the oracle on the exported state, energies against the CUDA-core path."""
    h, g = random_integrals(25, make_rng(MASTER_SEED + 11))
    ham = jw_molecular_hamiltonian(h, g)
    tmpl = uccsd_template(50, 10, max_excitations=60)
    theta = make_rng(MASTER_SEED + 21).uniform(-0.05, 0.05, tmpl.n_params)
    gates = tmpl.bind(theta)
    simt, tc = _pair(mps, ctx, 50, hf_bits(50, 10), gates, 128, 1e-5)
    rng = make_rng(MASTER_SEED + 320)
    idx = np.unique(np.concatenate([rng.choice(ham.n_terms, 300, replace=False),
                                    np.argsort(-np.abs(ham.coeffs))[:60]]))
    err_simt, e_simt = _errors(mps, ctx, simt, ham, idx)
    err_tc, e_tc = _errors(mps, ctx, tc, ham, idx)
    assert err_tc <= 1e-6 and err_tc <= max(3 * err_simt, 2e-7), (err_tc, err_simt)
    if list(simt.bond_dims()) == list(tc.bond_dims()):
        assert abs(e_tc - e_simt) <= 1e-5 * float(np.sum(np.abs(ham.coeffs)))
