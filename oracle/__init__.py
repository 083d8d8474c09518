"""FP64 CPU oracle of the MPS circuit simulation and Pauli-sum energy.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package: it is
used by ``tests/``, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg
of ``bench.py``.  It shares no code with the CUDA path; the only common
module is the seeded input generator ``paper_2303_03681_gb300.inputs``, which
holds no MPS arithmetic.

Contents (each function cites the passage of arXiv:2303.03681 it follows):

* ``mps``         - right-canonical MPS, one- and two-qubit gates with the
                    Hastings update and SVD truncation, expectation values by
                    Eq. (expec1)/(expec2), the Pauli-sum energy, and a second
                    canonical-form-free route by full transfer contraction.
* ``svd_jacobi``  - the one-sided Jacobi SVD of Algorithm 1 (complex, FP64).
* ``dense``       - brute-force dense statevector simulation (small n).
* ``fock``        - occupation-number-basis Hamiltonian, dense JW ladder
                    operators and the closed-form Hartree-Fock energy.
* ``rdm``         - 1- and 2-RDMs of a statevector by their definition
                    (ladder operators on occupation bit strings), their
                    spin-summed forms and the RDM energy (Methods, "The DMET
                    method").

Pins (tests/test_oracle_*.py, tests/test_rdm.py, all ``-m "not gpu"``):
dense statevector at uncapped bond dimension, the Hartree-Fock determinant
energy, the occupation-basis Hamiltonian, LAPACK singular values,
canonical-form and norm invariants, product-state expectation values, expm
of each UCCSD generator, the Hartree-Fock RDMs, trace and partial-trace
identities of the RDMs, and the RDM energy against the Pauli-sum energy.
Truncation (the rank rule and the renormalisation) is pinned by the dense
Schmidt truncation: one truncated gate on an exact state gives the best
rank-k approximation across that cut (Eckart-Young).  A sequence of
truncations has no closed form; there the oracle is checked through its
invariants (canonical form, unit norm, 1 - F <= 2 x discarded weight).
"""
