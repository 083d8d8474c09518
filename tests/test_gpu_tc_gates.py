"""GPU parity of the split-product tensor-core gate contractions.

MPS_PREC_TF32X3 and MPS_PREC_BF16X3 run the theta contraction C = Q (B_q
B_{q+1}) and B~_q = C V^dagger (Methods, "MPS algorithm for quantum circuit
simulation", Eqs. tildeC and Bl) as TMA-fed tcgen05 GEMMs whose real products
are sums of three piece products (hi*hi + hi*lo + lo*hi).  Each run is
compared with the FP64 oracle on the same circuit and with the complex64
CUDA-core path (MPS_PREC_FP32), on brickworks whose thetas span one to four
128-row tiles and ragged 64-column tiles (chi = 200).

Bars.  TF32 pieces keep 22 bits of every operand value, so TF32X3 is held to
the complex64 CUDA-core bars: 1 - F <= 1e-9 + 4 dw and per-string errors at
most 3x those of the CUDA-core path (or 2e-7).  BF16 pieces keep 16 bits
(relative 2^-17 per value), so a contraction carries about 1e-5 relative
error and BF16X3 is held to 1 - F <= 1e-6 + 4 dw and 1e-4 per string.
MPS_PREC_AUTO keeps these small bond capacities (< 256) on the CUDA cores, so
it must equal MPS_PREC_FP32 bit for bit.
"""

import numpy as np
import pytest

from gpu_helpers import to_oracle
from oracle import mps as om
from paper_2303_03681_gb300.inputs import MASTER_SEED, brickwork_circuit, make_rng, random_local_pauli_sum

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mps():
    from paper_2303_03681_gb300 import mps as m

    return m


@pytest.fixture(scope="module")
def ctx(mps):
    return mps.Context(0)


def _run(mps, ctx, n, circ, chi, trunc, precision):
    st = mps.State(ctx, n, None, chi_max=chi, precision=precision, trunc_rel=trunc, svd_fp64=1)
    rep = st.apply_gates(circ)
    assert rep["svd_not_converged"] == 0
    return st, rep


def _string_errors(mps, ctx, st, ham, ref):
    vals = st.expectations(mps.Hamiltonian(ctx, ham))
    want = np.array([om.expect_pauli(ref, row) for row in ham.ops])
    return float(np.max(np.abs(vals - want)))


@pytest.mark.parametrize("n,layers,chi", [(14, 10, 128), (16, 12, 200), (18, 12, 256)])
def test_split_products_match_oracle(mps, ctx, n, layers, chi):
    circ = brickwork_circuit(n, layers, make_rng(MASTER_SEED + 400 + n))
    ham = random_local_pauli_sum(n, 120, make_rng(MASTER_SEED + 401 + n))
    trunc = 1e-5
    ref = om.run_circuit(n, None, circ, chi_max=chi, eps_rel=trunc)
    simt, rep_s = _run(mps, ctx, n, circ, chi, trunc, "fp32")
    err_simt = _string_errors(mps, ctx, simt, ham, ref)
    B_simt, _ = simt.export()
    for precision, f_bar, s_bar in (("tf32x3", 1e-9, None), ("bf16x3", 1e-6, 1e-4)):
        st, rep = _run(mps, ctx, n, circ, chi, trunc, precision)
        got = to_oracle(st)
        dw = max(rep["discarded_weight"], ref.stats.discarded_weight)
        f = om.fidelity(got, ref)
        err = _string_errors(mps, ctx, st, ham, ref)
        B, _ = st.export()
        differs = any(a.shape != b.shape or not np.array_equal(a, b) for a, b in zip(B, B_simt))
        print(f"\n{precision} n={n} chi={chi}: 1-F={1 - f:.3e} dw={dw:.3e} max|d<P>|={err:.3e} "
              f"(CUDA cores {err_simt:.3e}) chi={max(st.bond_dims())}/{max(ref.bond_dims())}")
        assert differs, "the split-product path produced the CUDA-core result bit for bit: it did not run"
        assert 1 - f <= f_bar + 4 * dw
        if s_bar is None:
            assert err <= max(3 * err_simt, 2e-7), (err, err_simt)
        else:
            assert err <= s_bar


def test_auto_keeps_small_bonds_on_cuda_cores(mps, ctx):
    n, chi = 12, 64
    circ = brickwork_circuit(n, 8, make_rng(MASTER_SEED + 420))
    a, _ = _run(mps, ctx, n, circ, chi, 1e-5, "auto")
    b, _ = _run(mps, ctx, n, circ, chi, 1e-5, "fp32")
    Ba, La = a.export()
    Bb, Lb = b.export()
    assert all(np.array_equal(x, y) for x, y in zip(Ba, Bb))
    assert all(np.array_equal(x, y) for x, y in zip(La, Lb))


def test_split_products_through_vqe_eval_and_graphs(mps, ctx):
    """The tensor-core contractions inside a captured circuit graph, replayed:
    the same energies as host launches, and near the CUDA-core path."""
    from paper_2303_03681_gb300.inputs import CircuitTemplate

    n, chi = 14, 128
    tmpl = CircuitTemplate.from_gates(brickwork_circuit(n, 10, make_rng(MASTER_SEED + 430)))
    ham = random_local_pauli_sum(n, 80, make_rng(MASTER_SEED + 431))
    out = {}
    for graphs in (True, False):
        c = mps.Context(0)
        c.set_graphs(graphs)
        C, H = mps.Circuit(c, tmpl), mps.Hamiltonian(c, ham)
        st = mps.State(c, n, None, chi_max=chi, precision="tf32x3", trunc_rel=1e-5, svd_fp64=1)
        e, status = mps.vqe_eval(c, [(st, C, H, np.zeros(0), None)] * 2)
        assert list(status) == [0, 0]
        out[graphs] = e
    assert np.array_equal(out[True], out[False])
    assert out[True][0] == out[True][1]
    ref = om.energy(om.run_circuit(n, None, tmpl.bind(np.zeros(0)), chi_max=chi, eps_rel=1e-5), ham)
    assert abs(out[True][0] - ref) <= 1e-4
