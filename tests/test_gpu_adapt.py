"""The windowed qubit-ADAPT ansatz on the GPU (Methods, "The wave function
ansatz for hydrogen chain simulations").

Pool gradients come from ObservableGradients (one energy-kernel pass over the
commutator product strings plus one row-sum launch, mps_observables_eval) and
the re-optimisation energies from BatchedEnergy (vqe_eval_batch), both on
complex128 states at untruncated bond dimension.  The same loop driven by
the dense-statevector oracle (the oracle's gradient rows and energies) must
choose the same strings with energies equal to rounding, and H2/STO-3G must
reach the full-CI energy.
"""

import numpy as np
import pytest

from test_adapt import dense_gradients
from test_vqe_loop import DenseEnergy, h2_sto3g, sector_ground_energy
from paper_2303_03681_gb300.adapt import ObservableGradients, qubit_adapt
from paper_2303_03681_gb300.inputs import MASTER_SEED, hf_bits, jw_molecular_hamiltonian, make_rng, random_integrals
from paper_2303_03681_gb300.inputs.circuits import pauli_product_template, windowed_gsd_pool
from paper_2303_03681_gb300.vqe import BatchedEnergy, sequential_minimize

pytestmark = pytest.mark.gpu


def _gpu_loop(ham, pool, bits, n_qubits, chi, **kw):
    from paper_2303_03681_gb300 import mps

    ctx = mps.Context(0)
    grads = ObservableGradients(ctx, ham, pool, bits, chi_max=chi, precision="fp64")
    made = []

    def energy_factory(tmpl):
        e = BatchedEnergy(tmpl, ham, bits, slots=4, chi_max=chi, precision="fp64")
        made.append(e)
        return e

    res = qubit_adapt(pool, n_qubits, grads, energy_factory, **kw)
    for e in made:
        e.close()
    return res, grads


def test_gpu_pool_gradients_equal_the_oracle_rows():
    n_orb, n_e = 4, 4
    h, g = random_integrals(n_orb, make_rng(MASTER_SEED + 450))
    ham = jw_molecular_hamiltonian(h, g)
    bits = hf_bits(2 * n_orb, n_e)
    pool = windowed_gsd_pool(n_orb)
    from paper_2303_03681_gb300 import mps

    grads = ObservableGradients(mps.Context(0), ham, pool, bits, chi_max=16, precision="fp64")
    chosen = [3, 11, 0]
    tmpl = pauli_product_template(2 * n_orb, pool, chosen)
    theta = make_rng(MASTER_SEED + 451).uniform(-0.4, 0.4, len(chosen))
    want = dense_gradients(ham, pool, bits)(tmpl, theta)
    got = grads(tmpl, theta)
    assert np.max(np.abs(got - want)) <= 1e-10


def test_gpu_adapt_follows_the_oracle_loop():
    n_orb, n_e = 4, 4
    h, g = random_integrals(n_orb, make_rng(MASTER_SEED + 452))
    ham = jw_molecular_hamiltonian(h, g)
    bits = hf_bits(2 * n_orb, n_e)
    pool = windowed_gsd_pool(n_orb)
    kw = dict(max_ops=4, grad_tol=1e-8, optimizer=sequential_minimize, max_sweeps=4, tol=1e-10)
    gpu, _ = _gpu_loop(ham, pool, bits, 2 * n_orb, 16, **kw)
    grads = dense_gradients(ham, pool, bits)
    ref = qubit_adapt(pool, 2 * n_orb, grads, lambda t: DenseEnergy(t, ham, bits), **kw)
    # the first three choices have a unique largest gradient; at the fourth,
    # two spin-partner strings tie exactly (|g| equal to all digits) and
    # rounding picks one: the GPU's pick must attain the oracle's maximum
    assert gpu.chosen[:3] == ref.chosen[:3]
    assert np.max(np.abs(np.array(gpu.energies[:3]) - np.array(ref.energies[:3]))) <= 1e-9
    assert np.max(np.abs(np.array(gpu.max_gradients) - np.array(ref.max_gradients))) <= 1e-9
    ref3 = qubit_adapt(pool, 2 * n_orb, grads, lambda t: DenseEnergy(t, ham, bits), **dict(kw, max_ops=3))
    g3 = np.abs(grads(pauli_product_template(2 * n_orb, pool, ref3.chosen), ref3.theta))
    assert abs(g3[gpu.chosen[3]] - g3.max()) <= 1e-9
    assert abs(gpu.energies[3] - ref.energies[3]) <= 1e-6  # symmetric partners: equal energies after re-optimising
    assert gpu.energy >= sector_ground_energy(ham, n_e) - 1e-10


def test_gpu_adapt_reaches_h2_full_ci():
    ham = h2_sto3g()
    bits = hf_bits(4, 2)
    pool = windowed_gsd_pool(2)
    res, _ = _gpu_loop(ham, pool, bits, 4, 4, max_ops=4, grad_tol=1e-7, tol=1e-13)
    assert res.converged and len(res.chosen) <= 3
    assert abs(res.energy - sector_ground_energy(ham, 2)) <= 1e-9
