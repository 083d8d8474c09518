"""Stored oracle energies of the bench workloads (tests/golden/*_oracle.json,
written by tests/golden/make_oracle_energies.py) and the bench's lookup of
them (CPU only)."""

import json
import os
import sys
import types

import numpy as np

from oracle import dense as od
from paper_2303_03681_gb300.inputs import MASTER_SEED, brickwork_circuit, hf_bits, make_rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
if GOLDEN not in sys.path:  # the script that writes the records
    sys.path.insert(0, GOLDEN)


def _rec(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_c1_record_equals_the_dense_statevector_energy():
    """C1 is untruncated (chi 64 on 12 qubits), so its stored MPS-oracle
    energy must equal the brute-force dense energy."""
    import make_oracle_energies as m

    rec = _rec("c1_brickwork12_oracle.json")
    w = m.workload("c1")
    psi = od.run(12, hf_bits(12, 6), brickwork_circuit(12, 8, make_rng(MASTER_SEED + 1)))
    assert abs(od.energy(psi, w["ham"]) - rec["oracle_energy"]) <= 1e-10
    assert rec["n_terms"] == w["ham"].n_terms == 1819 and rec["oracle_discarded_weight"] == 0.0


def test_bench_oracle_check_matches_its_record():
    import bench

    rec = _rec("c1_brickwork12_oracle.json")
    w = bench.build_workload("c1", types.SimpleNamespace(precision=None), 0)
    seen = []

    class FakeMps:
        MPS_ENOTCONV = 5

        @staticmethod
        def vqe_eval_batch(reqs):
            seen.append(reqs)
            return np.array([rec["oracle_energy"] + 2e-12]), np.array([0], dtype=np.int32)

    class FakeState:
        def report(self):
            return {"discarded_weight": 0.0, "svd_not_converged": 0}

    chk = bench.oracle_check(FakeMps, FakeState(), None, None, w, w["trunc"])
    assert chk["reference"] == os.path.join("tests", "golden", "c1_brickwork12_oracle.json")
    assert abs(chk["abs_error_ha"] - 2e-12) <= 1e-15 and chk["energy_oracle"] == rec["oracle_energy"]
    assert chk["within_tol"] and chk["tolerance_ha"] == 1e-6
    assert len(seen) == 1 and seen[0][0][3].shape == (0,)  # C1 has no angles
    assert bench.oracle_check(FakeMps, FakeState(), None, None, w, 1e-3) is None  # other truncation: no record
