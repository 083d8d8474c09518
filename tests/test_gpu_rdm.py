"""Reduced density matrices on the GPU (mps_observables_eval) against the
oracle's (ladder operators on the dense statevector).

complex128 states: every element within 1e-10; complex64 states: within
1e-5 (storage rounding of the site tensors).  The spin-summed RDMs give back
the state's energy (E = sum h D + 1/2 sum (pq|rs) d) and electron count.
"""

import numpy as np
import pytest

from oracle import dense as od
from oracle import mps as om
from oracle import rdm as orr
from paper_2303_03681_gb300.inputs import (MASTER_SEED, brickwork_circuit, hf_bits, jw_molecular_hamiltonian,
                                           make_rng, random_integrals, uccsd_template)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mps():
    from paper_2303_03681_gb300 import mps as m

    return m


@pytest.fixture(scope="module")
def ctx(mps):
    return mps.Context(0)


def test_uccsd_rdms_and_energy_identity(mps, ctx):
    from paper_2303_03681_gb300.rdm import KINDS, RDM

    n_orb, n_e = 4, 4
    n_so = 2 * n_orb
    rng = make_rng(MASTER_SEED + 93)
    h, g = random_integrals(n_orb, rng)
    ham = jw_molecular_hamiltonian(h, g)
    tmpl = uccsd_template(n_so, n_e)
    bits = hf_bits(n_so, n_e)
    gates = tmpl.bind(rng.uniform(-0.4, 0.4, tmpl.n_params))
    st = mps.State(ctx, n_so, bits, chi_max=16, precision="fp64")
    st.apply_gates(gates)
    rdm = RDM(ctx, n_so, KINDS)
    got = rdm(st)
    psi = od.run(n_so, bits, gates)
    g1, g2 = orr.one_rdm(psi, n_so), orr.two_rdm(psi, n_so)
    D, d = orr.spatial_rdms(g1, g2)
    for k, ref in (("1rdm", g1), ("2rdm", g2), ("D", D), ("d", d)):
        assert np.max(np.abs(got[k] - ref)) <= 1e-10, k
    e = st.energy(mps.Hamiltonian(ctx, ham))
    assert abs(orr.rdm_energy(h, g, got["D"], got["d"]) - e) <= 1e-10
    assert abs(np.trace(got["D"]) - n_e) <= 1e-10
    again = rdm(st)  # the per-state output buffer is reused
    assert all(np.array_equal(again[k], got[k]) for k in KINDS)


def test_brickwork_12q_one_body_rdms(mps, ctx):
    """A complex 12-qubit state at chi 64 (the C1 circuit): complex 1-RDMs."""
    from paper_2303_03681_gb300.rdm import RDM

    n = 12
    circ = brickwork_circuit(n, 8, make_rng(MASTER_SEED + 1))
    ref = om.run_circuit(n, None, circ, chi_max=64)
    psi = om.to_statevector(ref)
    st = mps.State(ctx, n, None, chi_max=64, precision="fp64")
    st.apply_gates(circ)
    got = RDM(ctx, n, ("1rdm", "D"))(st)
    g1 = orr.one_rdm(psi, n)
    D = g1[0::2, 0::2] + g1[1::2, 1::2]
    assert np.max(np.abs(got["1rdm"] - g1)) <= 1e-10
    assert np.max(np.abs(got["D"] - D)) <= 1e-10
    assert np.max(np.abs(g1.imag)) > 1e-3


def test_complex64_state(mps, ctx):
    from paper_2303_03681_gb300.rdm import RDM

    n = 10
    circ = brickwork_circuit(n, 6, make_rng(MASTER_SEED + 94))
    psi = od.run(n, None, circ)
    st = mps.State(ctx, n, None, chi_max=32, precision="fp32", trunc_rel=1e-5, svd_fp64=True)
    st.apply_gates(circ)
    got = RDM(ctx, n, ("1rdm",))(st)
    assert np.max(np.abs(got["1rdm"] - orr.one_rdm(psi, n))) <= 1e-5


def test_observables_reject_inconsistent_rows(mps, ctx):
    from paper_2303_03681_gb300.inputs.hamiltonian import PauliSum

    strings = mps.Hamiltonian(ctx, PauliSum(4, np.array([[0, 0, 0, 0], [3, 0, 0, 0]], np.uint8), np.ones(2)))
    for row_ptr, cols in [([0, 1], [2]), ([0, 2, 1], [0, 1]), ([1, 2], [0, 1]), ([0, 1], [-1])]:
        with pytest.raises(mps.MpsError) as ei:
            mps.Observables(strings, row_ptr, cols, np.ones(len(cols)))
        assert ei.value.status == mps.MPS_EINVAL
    st = mps.State(ctx, 4, np.array([1, 0, 0, 0], np.uint8), chi_max=4)
    obs = mps.Observables(strings, [0, 2, 2], [0, 1], np.array([0.5, -0.5]))  # n_0 = (1 - Z_0) / 2, empty row
    assert np.array_equal(st.observables(obs), np.array([1.0, 0.0], complex))
    wrong = mps.State(ctx, 6, None, chi_max=4)
    with pytest.raises(mps.MpsError) as ei:
        wrong.observables(obs)
    assert ei.value.status == mps.MPS_EINVAL
