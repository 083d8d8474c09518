"""The variational loop on the GPU: the optimisers of ``vqe`` driven by
batched (vqe_eval_batch) and served (vqe_submit / vqe_poll) energies.

complex128 states at untruncated bond dimension: the GPU energies equal the
FP64 oracle's to rounding, so the loop follows the oracle-driven loop, the
shift-rule gradient matches the oracle's to 1e-10, and H2/STO-3G reaches the
textbook full-CI energy.
"""

import numpy as np
import pytest

from test_vqe_loop import DenseEnergy, OracleEnergy, h2_sto3g, sector_ground_energy, small_molecule
from paper_2303_03681_gb300.inputs import MASTER_SEED, hf_bits, make_rng, uccsd_template
from paper_2303_03681_gb300.vqe import (BatchedEnergy, ServedEnergy, bfgs_minimize, sequential_minimize,
                                        shift_gradient)

pytestmark = pytest.mark.gpu


def test_batched_loop_reaches_h2_full_ci():
    ham = h2_sto3g()
    tmpl, bits = uccsd_template(4, 2), hf_bits(4, 2)
    gpu = BatchedEnergy(tmpl, ham, bits, slots=4, chi_max=4, precision="fp64")
    e_fci = sector_ground_energy(ham, 2)
    res = sequential_minimize(gpu, np.zeros(tmpl.n_params), tol=1e-12)
    assert res.converged and abs(res.energy - e_fci) <= 1e-9
    res = bfgs_minimize(gpu, np.zeros(tmpl.n_params), gtol=1e-9)
    assert res.converged and abs(res.energy - e_fci) <= 1e-9
    theta = make_rng(MASTER_SEED + 80).uniform(-0.5, 0.5, tmpl.n_params)
    ref = OracleEnergy(tmpl, ham, bits, chi_max=4)
    assert np.max(np.abs(shift_gradient(gpu, theta) - shift_gradient(ref, theta))) <= 1e-10
    gpu.close()


def test_batched_loop_follows_the_oracle_loop():
    """Same optimiser, GPU energies vs dense-statevector energies: the energy
    trajectories agree to rounding and stay above the exact sector energy.

    The angles are not unique: moving two coupled single-excitation angles
    by pi each can leave E unchanged, so a one-angle model can have two equal
    minima and rounding picks one.  The test therefore compares the energies
    and checks the GPU's angles by the oracle's energy at them."""
    ham, tmpl, bits = small_molecule(3, 2, 81)
    gpu = BatchedEnergy(tmpl, ham, bits, slots=4, chi_max=8, precision="fp64")
    ref = DenseEnergy(tmpl, ham, bits)
    a = sequential_minimize(gpu, np.zeros(tmpl.n_params), max_sweeps=4, tol=0.0)
    b = sequential_minimize(ref, np.zeros(tmpl.n_params), max_sweeps=4, tol=0.0)
    assert np.max(np.abs(np.array(a.history) - np.array(b.history))) <= 1e-9
    assert abs(ref(a.theta[None])[0] - a.energy) <= 1e-10
    assert a.energy >= sector_ground_energy(ham, 2) - 1e-10
    assert a.n_evals == b.n_evals and a.n_batches == b.n_batches
    gpu.close()


def test_served_loop_matches_batched():
    """Energies through the serving engine equal the batched ones (the same
    kernels on the same data), and the loop converges through it."""
    ham = h2_sto3g()
    tmpl, bits = uccsd_template(4, 2), hf_bits(4, 2)
    cfg = dict(chi_max=4, precision="fp64")
    gpu = BatchedEnergy(tmpl, ham, bits, slots=4, **cfg)
    srv = ServedEnergy(tmpl, ham, bits, max_slots=2, trunc_rel=0.0, svd_fp64=True, **cfg)
    thetas = make_rng(MASTER_SEED + 82).uniform(-1.0, 1.0, (8, tmpl.n_params))
    assert np.max(np.abs(srv(thetas) - gpu(thetas))) <= 1e-12
    res = sequential_minimize(srv, np.zeros(tmpl.n_params), tol=1e-12)
    assert res.converged and abs(res.energy - sector_ground_energy(ham, 2)) <= 1e-9
    assert len(srv.latencies_ms) == 8 + res.n_evals and min(srv.latencies_ms) > 0
    srv.close()
    gpu.close()
