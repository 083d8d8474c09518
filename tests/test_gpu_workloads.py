"""GPU parity at the benchmark's full sizes (C2: 50 qubits, chi_max = 128,
571,876-term Hamiltonian), in the launch configuration bench.py times.

The oracle cannot evaluate all 571,876 strings in test time, so the energy is
checked on sampled outputs it computes one by one: per-string expectation
values on an independent oracle run of the same circuit, plus the state
fidelity, norm and canonical-form properties that hold at any size.
"""

import numpy as np
import pytest

from gpu_helpers import to_oracle
from oracle import mps as om
from paper_2303_03681_gb300.inputs import (MASTER_SEED, hf_bits, jw_molecular_hamiltonian, make_rng,
                                           random_integrals, uccsd_template)

pytestmark = pytest.mark.gpu

N_ORB, N_E, CHI, TRUNC = 25, 10, 128, 1e-5


@pytest.fixture(scope="module")
def c2():
    h, g = random_integrals(N_ORB, make_rng(MASTER_SEED + 11))
    return jw_molecular_hamiltonian(h, g)


@pytest.mark.parametrize("n_exc,svd", [(40, "fp64"), (100, "fp32")])
def test_c2_prefix_matches_oracle(c2, n_exc, svd):
    from paper_2303_03681_gb300 import mps

    ham = c2
    tmpl = uccsd_template(2 * N_ORB, N_E, max_excitations=n_exc)
    bits = hf_bits(2 * N_ORB, N_E)
    theta = make_rng(MASTER_SEED + 21).uniform(-0.05, 0.05, tmpl.n_params)
    ctx = mps.Context(0)
    st = mps.State(ctx, 2 * N_ORB, bits, chi_max=CHI, precision="fp32", trunc_rel=TRUNC, svd_fp64=(svd == "fp64"))
    C = mps.Circuit(ctx, tmpl)
    H = mps.Hamiltonian(ctx, ham)
    st.apply_circuit(C, theta)
    vals = st.expectations(H)
    e_gpu = st.energy(H)
    assert abs(e_gpu - float(np.dot(ham.coeffs, vals))) <= 1e-9 * max(1.0, abs(e_gpu))

    ref = om.run_circuit(2 * N_ORB, bits, tmpl.bind(theta), chi_max=CHI, eps_rel=TRUNC)
    got = to_oracle(st)
    assert om.fidelity(got, ref) >= 1 - 1e-8
    assert abs(om.norm_full(got) - 1.0) <= 1e-5
    rng = make_rng(MASTER_SEED + 22)
    sample = np.unique(np.concatenate([rng.choice(ham.n_terms, 600, replace=False),
                                       np.argsort(-np.abs(ham.coeffs))[:100]]))
    want = np.array([om.expect_pauli(ref, ham.ops[k]) for k in sample])
    assert np.max(np.abs(vals[sample] - want)) <= 2e-6
    # energy difference estimated from the sample, scaled to all terms
    est = np.abs(np.dot(ham.coeffs[sample], vals[sample] - want)) * np.sqrt(ham.n_terms / sample.size)
    assert est <= 1e-5
