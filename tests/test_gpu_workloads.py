"""GPU parity at the benchmark's full sizes (C2: 50 qubits, chi_max = 128,
571,876-term Hamiltonian), in the launch configuration bench.py times.

The oracle cannot evaluate all 571,876 strings in test time, so the energy is
checked on outputs it computes one by one: per-string expectation values on
an independent oracle run of the same circuit, an importance-sampled estimate
of the energy difference, and the state fidelity, norm and canonical form,
which hold at any size.

Tolerance.  Both sides truncate at the same chi_max and eps_rel, but a
singular value within rounding of the eps_rel threshold can be kept on one
side and dropped on the other; the two truncated states then differ by about
the discarded weight dw.  The bar is 1 - F <= 1e-8 + 4 dw, and per string
|<P>_gpu - <P>_oracle| <= 2 sqrt(1 - F) + 1e-6 (|<a|P|a> - <b|P|b>| <= 2 ||a - b||).
"""

import numpy as np
import pytest

from gpu_helpers import to_oracle
from oracle import mps as om
from paper_2303_03681_gb300.inputs import (MASTER_SEED, hf_bits, jw_molecular_hamiltonian, make_rng,
                                           random_integrals, uccsd_template)

pytestmark = pytest.mark.gpu

N_ORB, N_E, CHI = 25, 10, 128


@pytest.fixture(scope="module")
def c2():
    h, g = random_integrals(N_ORB, make_rng(MASTER_SEED + 11))
    return jw_molecular_hamiltonian(h, g)


@pytest.mark.parametrize("n_exc,svd,trunc", [(40, "fp64", 1e-5), (100, "fp32", 1e-5), (140, "fp32", 1e-5)])
def test_c2_prefix_matches_oracle(c2, n_exc, svd, trunc):
    from paper_2303_03681_gb300 import mps

    ham = c2
    tmpl = uccsd_template(2 * N_ORB, N_E, max_excitations=n_exc)
    bits = hf_bits(2 * N_ORB, N_E)
    theta = make_rng(MASTER_SEED + 21).uniform(-0.05, 0.05, tmpl.n_params)
    ctx = mps.Context(0)
    st = mps.State(ctx, 2 * N_ORB, bits, chi_max=CHI, precision="fp32", trunc_rel=trunc, svd_fp64=(svd == "fp64"))
    C = mps.Circuit(ctx, tmpl)
    H = mps.Hamiltonian(ctx, ham)
    st.apply_circuit(C, theta)
    vals = st.expectations(H)
    e_gpu = st.energy(H)
    rep = st.report()
    assert abs(e_gpu - float(np.dot(ham.coeffs, vals))) <= 1e-9 * max(1.0, abs(e_gpu))

    ref = om.run_circuit(2 * N_ORB, bits, tmpl.bind(theta), chi_max=CHI, eps_rel=trunc)
    got = to_oracle(st)
    f = om.fidelity(got, ref)
    dw = max(ref.stats.discarded_weight, rep["discarded_weight"])
    rng = make_rng(MASTER_SEED + 22)
    sample = np.unique(np.concatenate([rng.choice(ham.n_terms, 400, replace=False),
                                       np.argsort(-np.abs(ham.coeffs))[:100]]))
    want = np.array([om.expect_pauli(ref, ham.ops[k]) for k in sample])
    diff = vals[sample] - want
    # importance-sampled energy difference: k ~ |c_k| / sum |c|
    w = np.abs(ham.coeffs) / np.sum(np.abs(ham.coeffs))
    ks = rng.choice(ham.n_terms, 300, p=w)
    dk = np.array([vals[k] - om.expect_pauli(ref, ham.ops[k]) for k in ks])
    est = np.sum(np.abs(ham.coeffs)) * np.mean(np.sign(ham.coeffs[ks]) * dk)
    est_err = np.sum(np.abs(ham.coeffs)) * np.std(np.sign(ham.coeffs[ks]) * dk) / np.sqrt(ks.size)
    print(f"\nC2 prefix {n_exc} exc, svd {svd}, eps {trunc}: 1-F={1 - f:.3e} dw_gpu={rep['discarded_weight']:.3e} "
          f"dw_oracle={ref.stats.discarded_weight:.3e} chi_gpu={rep['max_chi']} chi_oracle={ref.stats.max_chi} "
          f"max|d<P>|={np.max(np.abs(diff)):.3e} dE~{est:.3e}+-{est_err:.1e} E_gpu={e_gpu:.9f}")
    assert 1 - f <= 1e-8 + 4 * dw
    assert abs(om.norm_full(got) - 1.0) <= 1e-5
    assert np.max(np.abs(diff)) <= 2 * np.sqrt(max(1 - f, 0.0)) + 1e-6
