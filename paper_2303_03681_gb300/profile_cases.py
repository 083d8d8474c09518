"""Small workloads for single-kernel ncu captures.

  python paper_2303_03681_gb300/profile_cases.py tc      # tcgen05 environment GEMMs
  python paper_2303_03681_gb300/profile_cases.py svd64   # cluster Jacobi, every sweep in FP64
  python paper_2303_03681_gb300/profile_cases.py svdmix  # cluster Jacobi, FP32 then FP64 sweeps

Each case keeps the device footprint to a few hundred MB and the launch
count small, so that a ``--set full`` capture of one or two launches ends by
itself within a minute or two.

* ``tc``: 18-qubit Haar brickwork of 12 layers at chi_max 200, complex64
  storage, FP32 Jacobi, tensor-core environments; 300 random 1-, nearest-
  and next-nearest-site Pauli strings; three energy evaluations.
* ``svd64`` / ``svdmix``: 14-qubit brickwork of 10 layers at chi_max 64,
  complex64 storage, trunc_rel 1e-5.
"""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2303_03681_gb300 import mps  # noqa: E402
from paper_2303_03681_gb300.inputs import MASTER_SEED, brickwork_circuit, make_rng, random_local_pauli_sum  # noqa: E402


def main(what: str) -> None:
    ctx = mps.Context(0)
    if what in ("svd64", "svdmix"):
        circ = brickwork_circuit(14, 10, make_rng(MASTER_SEED + 12))
        st = mps.State(ctx, 14, None, chi_max=64, precision="fp32", trunc_rel=1e-5,
                       svd_fp64=2 if what == "svd64" else 1)
        print(st.apply_gates(circ))
    elif what == "tc":
        circ = brickwork_circuit(18, 12, make_rng(MASTER_SEED + 318))
        st = mps.State(ctx, 18, None, chi_max=200, precision="fp32", svd_fp64=0, tensor_cores=True)
        st.apply_gates(circ)
        ham = random_local_pauli_sum(18, 300, make_rng(MASTER_SEED + 319))
        H = mps.Hamiltonian(ctx, ham)
        for _ in range(3):
            print(st.energy(H))
    else:
        raise SystemExit(f"unknown case {what!r}: tc, svd64 or svdmix")
    ctx.synchronize()


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "tc")
