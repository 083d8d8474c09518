"""Writes FP64 oracle energies of the bench workloads at fixed angles, for
stating the GPU's error against the oracle at full size
(tests/golden/<workload>_oracle.json; bench.py reports |E_gpu - E_oracle|
for the record matching its workload and truncation).

* ``c2``: 25-orbital random integrals (seed MASTER_SEED + 11, 571,876 JW
  strings), UCCSD-style template of the 10-electron Hartree-Fock reference
  restricted to its first 100 excitations (10,760 two-qubit gates), angles
  U[-0.05, 0.05] from seed MASTER_SEED + 21, chi_max 128, eps_rel 1e-5.
  Tens of minutes on one host.
* ``c1``: 6-orbital random integrals (seed MASTER_SEED), 8-layer Haar
  brickwork on 12 qubits (seed MASTER_SEED + 1, no angles), Hartree-Fock
  reference with 6 electrons, chi_max 64, eps_rel 0.  Seconds.

Calls only the oracle (``oracle.mps``: LAPACK SVD, Eq. expec2 per string,
FP64) and the seeded input generators.  The per-string values <P_k> are
independent, so they are computed by a pool of processes (``spawn``) over
slices of the strings; the parent then forms sum_k c_k <P_k> in index order,
the order of ``oracle.mps.energy``, so the result equals a serial run's.

  python tests/golden/make_oracle_energies.py c2|c1 [processes]
"""

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import mps as om  # noqa: E402
from paper_2303_03681_gb300.inputs import (MASTER_SEED, CircuitTemplate, brickwork_circuit, hf_bits,  # noqa: E402
                                           jw_molecular_hamiltonian, make_rng, random_integrals, uccsd_template)


def workload(name: str):
    if name == "c2":
        n_exc = 100
        h, g = random_integrals(25, make_rng(MASTER_SEED + 11))
        tmpl = uccsd_template(50, 10, max_excitations=n_exc)
        return dict(workload=f"c2_uccsd_50q_chi128_first{n_exc}exc", ham=jw_molecular_hamiltonian(h, g), tmpl=tmpl,
                    bits=hf_bits(50, 10), chi=128, eps=1e-5, theta_seed=MASTER_SEED + 21, theta_range=[-0.05, 0.05],
                    integrals_seed=MASTER_SEED + 11, file="c2_uccsd50_first100exc_oracle.json")
    if name == "c1":
        h, g = random_integrals(6, make_rng(MASTER_SEED))
        tmpl = CircuitTemplate.from_gates(brickwork_circuit(12, 8, make_rng(MASTER_SEED + 1)))
        return dict(workload="c1_brickwork_12q_8layers_chi64", ham=jw_molecular_hamiltonian(h, g), tmpl=tmpl,
                    bits=hf_bits(12, 6), chi=64, eps=0.0, theta_seed=MASTER_SEED + 21, theta_range=[0.0, 0.0],
                    integrals_seed=MASTER_SEED, file="c1_brickwork12_oracle.json")
    raise SystemExit(f"unknown workload {name!r}: c2 or c1")


def _values(args):
    state, ops = args
    return [om.expect_pauli(state, row) for row in ops]


def energy_parallel(state, ham, processes: int) -> float:
    import multiprocessing as mp

    n = ham.n_terms
    step = max(1, -(-n // (8 * processes)))
    slices = [(state, ham.ops[lo: lo + step]) for lo in range(0, n, step)]
    # one BLAS thread per worker process (the contractions are small)
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    with mp.get_context("spawn").Pool(processes) as pool:
        vals = [v for part in pool.map(_values, slices) for v in part]
    return float(sum(c * v for c, v in zip(ham.coeffs, vals)))


def main(name: str, processes: int = 0) -> str:
    w = workload(name)
    tmpl, ham = w["tmpl"], w["ham"]
    lo, hi = w["theta_range"]
    theta = make_rng(w["theta_seed"]).uniform(lo, hi, tmpl.n_params)
    t0 = time.time()
    ref = om.run_circuit(tmpl.n_qubits, w["bits"], tmpl.bind(theta), chi_max=w["chi"], eps_rel=w["eps"])
    t1 = time.time()
    energy = energy_parallel(ref, ham, processes) if processes > 1 else om.energy(ref, ham)
    t2 = time.time()
    out = {
        "source": "written by tests/golden/make_oracle_energies.py from the FP64 oracle (oracle.mps)",
        "workload": w["workload"], "n_qubits": tmpl.n_qubits, "chi_max": w["chi"], "trunc_rel": w["eps"],
        "n_terms": int(ham.n_terms), "two_qubit_gates": int(tmpl.n_two_qubit),
        "integrals_seed": w["integrals_seed"], "theta_seed": w["theta_seed"], "theta_range": [lo, hi],
        "oracle_energy": energy,
        "oracle_discarded_weight": ref.stats.discarded_weight, "oracle_max_chi": ref.stats.max_chi,
        "oracle_seconds": {"gates": round(t1 - t0, 1), "energy": round(t2 - t1, 1),
                           "energy_processes": max(1, processes)},
    }
    path = os.path.join(HERE, w["file"])
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    return path


if __name__ == "__main__":
    print(main(sys.argv[1] if len(sys.argv) > 1 else "c2",
               int(sys.argv[2]) if len(sys.argv) > 2 else (os.cpu_count() or 1)))
