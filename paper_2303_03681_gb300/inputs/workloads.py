"""Seeded specifications of the multi-instance and large synthetic workloads.

Each function returns light-weight specs (sizes, seeds, bond-dimension caps);
``build()`` on a spec draws its circuit and Hamiltonian on demand, because a
full UCCSD template of a large fragment has hundreds of thousands of
excitations and is only ever built with an excitation cap.

* ``precision_instance`` (100 qubits, chi 512): Haar brickwork of 40 layers
  and 2,000 distinct 1-, nearest- and next-nearest-site Pauli strings with
  N(0, 1) coefficients.
* ``fragment_batch`` (256 uneven embedding fragments): qubits uniform over
  the even numbers 8..40, half filling (n_e = n_orb), chi uniform over
  {32, 64, 128, 256} clipped to 2^(n/2); UCCSD-style circuit and a
  random-integral Hamiltonian sized to the fragment's orbitals.
* ``serving_fleet``: 200 resident fragments, qubits uniform over the even
  numbers 10..100, chi_max uniform over {64, 128, 256, 512, 1024} clipped,
  plus one 1,000-qubit brickwork of 16 layers at chi 256 with 10,000
  distinct 1- and nearest-site Pauli strings.

Fragment k of a batch draws everything from ``instance_seed(offset + k)``.
"""

from dataclasses import dataclass

import numpy as np

from .circuits import CircuitTemplate, brickwork_circuit, uccsd_template
from .hamiltonian import hf_bits, jw_molecular_hamiltonian, random_integrals, random_local_pauli_sum
from .rng import MASTER_SEED, instance_seed, make_rng


@dataclass(frozen=True)
class FragmentSpec:
    """A UCCSD-style VQE fragment: n_qubits = 2 n_orb, n_e electrons."""

    index: int
    n_qubits: int
    n_electrons: int
    chi_max: int
    seed: int

    def build(self, max_excitations=None):
        """(template, Hamiltonian, HF bits); ``max_excitations`` caps the circuit."""
        n_orb = self.n_qubits // 2
        rng = make_rng(self.seed)
        h, g = random_integrals(n_orb, rng)
        ham = jw_molecular_hamiltonian(h, g)
        tmpl = uccsd_template(self.n_qubits, self.n_electrons, max_excitations=max_excitations)
        return tmpl, ham, hf_bits(self.n_qubits, self.n_electrons)

    def thetas(self, count: int, scale: float = 0.05, n_params=None):
        """Angles for ``count`` evaluations, U[-scale, scale]."""
        rng = make_rng(self.seed + 7_000_000)
        n = self.n_params() if n_params is None else int(n_params)
        return rng.uniform(-scale, scale, (count, n))

    def n_params(self) -> int:
        from .circuits import uccsd_excitations

        return len(uccsd_excitations(self.n_qubits, self.n_electrons))


@dataclass(frozen=True)
class BrickworkSpec:
    """A brickwork circuit with a 1D local Pauli sum."""

    n_qubits: int
    layers: int
    chi_max: int
    n_terms: int
    next_nearest: bool
    seed: int

    def build(self):
        """(template, Hamiltonian, None): the fixed circuit as a template."""
        circ = brickwork_circuit(self.n_qubits, self.layers, make_rng(self.seed))
        ham = random_local_pauli_sum(self.n_qubits, self.n_terms, make_rng(self.seed + 1),
                                     next_nearest=self.next_nearest)
        return CircuitTemplate.from_gates(circ), ham, None


def _clip_chi(chi: int, n_qubits: int) -> int:
    return int(min(chi, 2 ** (n_qubits // 2)))


def precision_instance(seed: int = MASTER_SEED + 30) -> BrickworkSpec:
    return BrickworkSpec(100, 40, 512, 2000, True, seed)


def fragment_batch(count: int = 256, offset: int = 1000):
    rng = make_rng(MASTER_SEED + 40)
    qubits = 2 * rng.integers(4, 21, count)  # 8..40, even
    chis = rng.choice([32, 64, 128, 256], count)
    return [FragmentSpec(k, int(q), int(q) // 2, _clip_chi(int(c), int(q)), instance_seed(offset + k))
            for k, (q, c) in enumerate(zip(qubits, chis))]


def serving_fleet(count: int = 200, offset: int = 2000):
    rng = make_rng(MASTER_SEED + 50)
    qubits = 2 * rng.integers(5, 51, count)  # 10..100, even
    chis = rng.choice([64, 128, 256, 512, 1024], count)
    frags = [FragmentSpec(k, int(q), int(q) // 2, _clip_chi(int(c), int(q)), instance_seed(offset + k))
             for k, (q, c) in enumerate(zip(qubits, chis))]
    big = BrickworkSpec(1000, 16, 256, 10_000, False, MASTER_SEED + 51)
    return frags, big
