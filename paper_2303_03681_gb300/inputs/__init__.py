"""Seeded synthetic input generators shared by the CUDA path and the oracle.

This subpackage produces the *inputs* of the hot path and nothing else:

* random molecular integrals and their Jordan-Wigner Pauli sums
  (second-quantised Hamiltonian of the paper's "Unitary coupled cluster"
  subsection, JW mapping as named there),
* random 1D Pauli sums on nearest and next-nearest neighbours,
* gate lists: Haar-random SU(4) brickwork circuits and UCCSD-style products
  of Pauli-string exponentials compiled to nearest-neighbour CNOT/SWAP
  ladders plus Rz (the paper's UCCSD-with-MPS subsection), with the
  variational angles bound separately.

It holds none of the matrix-product-state arithmetic (no contraction, SVD,
truncation or expectation value), so importing it never touches the CUDA
library or the oracle.
"""

from .rng import MASTER_SEED, make_rng, instance_seed
from .hamiltonian import (
    PauliSum,
    random_integrals,
    jw_molecular_hamiltonian,
    hf_bits,
    random_local_pauli_sum,
)
from .circuits import (
    GateList,
    CircuitTemplate,
    haar_su4,
    brickwork_circuit,
    uccsd_excitations,
    uccsd_template,
    pauli_exponential_template,
)

__all__ = [
    "MASTER_SEED",
    "make_rng",
    "instance_seed",
    "PauliSum",
    "random_integrals",
    "jw_molecular_hamiltonian",
    "hf_bits",
    "random_local_pauli_sum",
    "GateList",
    "CircuitTemplate",
    "haar_su4",
    "brickwork_circuit",
    "uccsd_excitations",
    "uccsd_template",
    "pauli_exponential_template",
]
