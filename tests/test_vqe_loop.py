"""The variational loop (UCC, Eq. ucc) on the CPU: its optimisers driven by
oracle and dense-statevector energies.

Pins: the one-angle energy of the compiled UCCSD circuits is exactly a
degree-2 trigonometric polynomial (checked through the FP64 MPS oracle at
off-grid points), the shift-rule gradient equals central finite differences
of the oracle energy, both optimisers reach the textbook H2/STO-3G full-CI
energy (UCCSD is exact for two electrons), and on a random 8-qubit molecule
the converged energy respects the variational bound of the 4-electron sector.
"""

import json
import os

import numpy as np
import pytest

from oracle import dense as od
from oracle import mps as om
from paper_2303_03681_gb300.inputs import (MASTER_SEED, hf_bits, jw_molecular_hamiltonian, make_rng,
                                           random_integrals, uccsd_template)
from paper_2303_03681_gb300.vqe import (bfgs_minimize, sequential_minimize, shift_gradient, trig_argmin,
                                        trig_coefficients, trig_value)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def h2_sto3g():
    with open(os.path.join(GOLDEN, "h2_sto3g.json")) as f:
        d = json.load(f)
    h = np.array(d["h"])
    g = np.zeros((2, 2, 2, 2))
    g[0, 0, 0, 0] = d["J11"]
    g[1, 1, 1, 1] = d["J22"]
    g[0, 0, 1, 1] = g[1, 1, 0, 0] = d["J12"]
    for idx in [(0, 1, 0, 1), (1, 0, 1, 0), (0, 1, 1, 0), (1, 0, 0, 1)]:
        g[idx] = d["K12"]
    return jw_molecular_hamiltonian(h, g)


def sector_ground_energy(ham, n_e):
    """Lowest eigenvalue of H restricted to n_e particles (brute force)."""
    H = od.hamiltonian_matrix(ham)
    n = ham.n_qubits
    idx = [i for i in range(1 << n) if bin(i).count("1") == n_e]
    return float(np.linalg.eigvalsh(H[np.ix_(idx, idx)])[0])


class DenseEnergy:
    """energy_batch from the dense statevector (oracle; small n)."""

    def __init__(self, tmpl, ham, bits):
        self.tmpl, self.bits = tmpl, bits
        self.H = od.hamiltonian_matrix(ham)

    def __call__(self, thetas):
        out = []
        for th in np.atleast_2d(thetas):
            psi = od.run(self.tmpl.n_qubits, self.bits, self.tmpl.bind(th))
            out.append(np.vdot(psi, self.H @ psi).real)
        return np.array(out)


class OracleEnergy:
    """energy_batch from the FP64 MPS oracle at untruncated bond dimension."""

    def __init__(self, tmpl, ham, bits, chi_max=64):
        self.tmpl, self.ham, self.bits, self.chi = tmpl, ham, bits, chi_max

    def __call__(self, thetas):
        return np.array([om.vqe_energy(self.tmpl, th, self.bits, self.ham, chi_max=self.chi)
                         for th in np.atleast_2d(thetas)])


def small_molecule(n_orb, n_e, seed_offset):
    h, g = random_integrals(n_orb, make_rng(MASTER_SEED + seed_offset))
    ham = jw_molecular_hamiltonian(h, g)
    return ham, uccsd_template(2 * n_orb, n_e), hf_bits(2 * n_orb, n_e)


def test_trig_fit_and_exact_minimum():
    rng = make_rng(MASTER_SEED + 70)
    grid = np.linspace(-np.pi, np.pi, 400001)
    for _ in range(50):
        coef = rng.normal(size=5)
        e5 = trig_value(coef, 2 * np.pi * np.arange(5) / 5)
        assert np.allclose(trig_coefficients(e5), coef, atol=1e-13, rtol=0)
        s = trig_argmin(coef)
        assert -np.pi < s <= np.pi
        assert trig_value(coef, s) <= trig_value(coef, grid).min() + 1e-12
    # degenerate models: constant, and first-harmonic only
    assert trig_value([1.0, 0, 0, 0, 0], trig_argmin([1.0, 0, 0, 0, 0])) == 1.0
    assert abs(trig_argmin([0.0, 1.0, 0.0, 0.0, 0.0]) - np.pi) < 1e-12


@pytest.mark.parametrize("which", ["single", "double"])
def test_one_angle_energy_is_a_degree_two_trig_polynomial(which):
    """exp(theta G) with G^3 = -G for every excitation generator, so E along
    one angle has frequencies 0, 1, 2 only: a fit through 5 points predicts
    the oracle energy at other angles to rounding."""
    ham, tmpl, bits = small_molecule(3, 2, 71)
    f = OracleEnergy(tmpl, ham, bits)
    rng = make_rng(MASTER_SEED + 72)
    theta = rng.uniform(-0.5, 0.5, tmpl.n_params)
    k = 0 if which == "single" else tmpl.n_params - 1  # singles come first, doubles last
    trial = np.repeat(theta[None], 8, axis=0)
    shifts = np.concatenate([2 * np.pi * np.arange(5) / 5, rng.uniform(-np.pi, np.pi, 3)])
    trial[:, k] += shifts
    e = f(trial)
    coef = trig_coefficients(e[:5])
    assert np.max(np.abs(trig_value(coef, shifts[5:]) - e[5:])) <= 1e-12
    assert abs(coef[3]) + abs(coef[4]) > 1e-6  # the second harmonic is really there


def test_shift_gradient_equals_finite_differences():
    ham, tmpl, bits = small_molecule(3, 2, 73)
    f = OracleEnergy(tmpl, ham, bits)
    theta = make_rng(MASTER_SEED + 74).uniform(-0.4, 0.4, tmpl.n_params)
    g = shift_gradient(f, theta)
    h = 1e-5
    fd = np.empty_like(g)
    for k in range(tmpl.n_params):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd[k] = (f(tp[None])[0] - f(tm[None])[0]) / (2 * h)
    assert np.max(np.abs(g - fd)) <= 1e-8
    assert np.max(np.abs(g)) > 1e-3


def test_sequential_minimisation_reaches_h2_full_ci():
    ham = h2_sto3g()
    tmpl, bits = uccsd_template(4, 2), hf_bits(4, 2)
    e_fci = sector_ground_energy(ham, 2)
    res = sequential_minimize(OracleEnergy(tmpl, ham, bits, chi_max=4), np.zeros(tmpl.n_params), tol=1e-12)
    assert res.converged
    assert abs(res.energy - e_fci) <= 1e-10
    assert res.n_evals == 1 + res.iterations * (4 * tmpl.n_params + 1)


def test_bfgs_with_shift_gradients_reaches_h2_full_ci():
    ham = h2_sto3g()
    tmpl, bits = uccsd_template(4, 2), hf_bits(4, 2)
    e_fci = sector_ground_energy(ham, 2)
    res = bfgs_minimize(OracleEnergy(tmpl, ham, bits, chi_max=4), np.zeros(tmpl.n_params), gtol=1e-9)
    assert res.converged
    assert abs(res.energy - e_fci) <= 1e-10


def test_random_molecule_is_variational_and_monotone():
    ham, tmpl, bits = small_molecule(4, 4, 75)
    f = DenseEnergy(tmpl, ham, bits)
    e_hf = float(f(np.zeros((1, tmpl.n_params)))[0])
    e_exact = sector_ground_energy(ham, 4)
    res = sequential_minimize(f, np.zeros(tmpl.n_params), max_sweeps=12, tol=1e-9)
    assert np.all(np.diff(res.history) <= 1e-12)  # exact coordinate steps never raise E
    assert e_exact - 1e-10 <= res.energy < e_hf - 1e-3
    # the measured energy at the returned angles is the reported one
    assert abs(f(res.theta[None])[0] - res.energy) <= 1e-12


def test_edge_cases():
    def const(thetas):
        return np.full(np.atleast_2d(thetas).shape[0], 2.5)

    res = sequential_minimize(const, np.zeros(0))  # no angles: the start and end-of-sweep energies only
    assert res.converged and res.energy == 2.5 and res.n_evals == 2 and res.theta.shape == (0,)
    assert np.array_equal(shift_gradient(const, np.zeros(3)), np.zeros(3))
    res = bfgs_minimize(const, np.zeros(3))  # flat: zero gradient at once
    assert res.converged and res.iterations == 1 and res.energy == 2.5
    with pytest.raises(ValueError):
        trig_coefficients(np.zeros(4))
    with pytest.raises(ValueError):
        sequential_minimize(lambda t: np.zeros(1), np.zeros(2))  # wrong number of energies
