"""Seeded specifications of the precision instance, the fragment batch and
the serving fleet (CPU): stated distributions, clipping of the bond
dimension to 2^(n/2), determinism, and built shapes."""

import numpy as np

from paper_2303_03681_gb300.inputs.workloads import fragment_batch, precision_instance, serving_fleet


def test_fragment_batch_distribution_and_determinism():
    specs = fragment_batch()
    assert len(specs) == 256 and specs == fragment_batch()
    q = np.array([s.n_qubits for s in specs])
    assert q.min() >= 8 and q.max() <= 40 and np.all(q % 2 == 0)
    assert len(set(q)) >= 15  # most of the 17 sizes occur
    for s in specs:
        assert s.n_electrons == s.n_qubits // 2
        assert s.chi_max in (16, 32, 64, 128, 256) and s.chi_max <= 2 ** (s.n_qubits // 2)
    assert len({s.seed for s in specs}) == 256


def test_small_fragment_builds():
    s = next(s for s in fragment_batch() if s.n_qubits == 8)
    tmpl, ham, bits = s.build()
    assert tmpl.n_qubits == ham.n_qubits == 8 and int(bits.sum()) == 4
    assert tmpl.n_params == s.n_params()
    th = s.thetas(3)
    assert th.shape == (3, tmpl.n_params) and np.all(np.abs(th) <= 0.05)
    tmpl2, ham2, _ = s.build(max_excitations=5)
    assert tmpl2.meta["n_excitations"] == 5 and np.array_equal(ham2.ops, ham.ops)


def test_precision_instance_and_fleet():
    p = precision_instance()
    tmpl, ham, bits = p.build()
    assert bits is None and tmpl.n_qubits == 100 and tmpl.n_two_qubit == 1980 and ham.n_terms == 2000
    spans = [np.nonzero(r)[0][-1] - np.nonzero(r)[0][0] for r in ham.ops]
    assert max(spans) == 2
    frags, big = serving_fleet()
    assert len(frags) == 200 and frags == serving_fleet()[0]
    q = np.array([f.n_qubits for f in frags])
    assert q.min() >= 10 and q.max() <= 100 and np.all(q % 2 == 0)
    assert all(f.chi_max <= min(1024, 2 ** (f.n_qubits // 2)) for f in frags)
    tmpl, ham, _ = big.build()
    assert tmpl.n_qubits == 1000 and tmpl.n_two_qubit == 8 * 500 + 8 * 499 and ham.n_terms == 10_000
    spans = [np.nonzero(r)[0][-1] - np.nonzero(r)[0][0] for r in ham.ops]
    assert max(spans) == 1
