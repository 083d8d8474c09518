"""mps_gate2_noalloc against the regular gate path and the oracle (GPU).

mps_gate2_noalloc exists for callers that cannot allocate device memory; it
applies one two-qubit gate to caller-owned device buffers using a fixed
scratch array inside the library.  This test applies the same two gates in a
row through it and through mps_apply_gates on an MPS with the same tensors (and the FP64
oracle's update of those tensors), and compares the gauge-invariant results: the new bond's singular values and
the two-site tensor B~_q B~_{q+1}, within the complex128 parity tolerance of
the other GPU tests (1e-10).  It runs last so that a failure here comes after
every other test, and it passes alone in a fresh process too: the entry
point's first call on the device does its own set-up.
"""

import ctypes

import numpy as np
import pytest

from oracle import mps as orc
from paper_2303_03681_gb300.inputs import brickwork_circuit, haar_su4, make_rng

pytestmark = pytest.mark.gpu


def _noalloc(lib):
    fn = lib.mps_gate2_noalloc
    P = ctypes.c_void_p
    fn.argtypes = [ctypes.c_int, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P, P, P, P, ctypes.c_int32,
                   ctypes.c_double, P]
    fn.restype = ctypes.c_int
    return fn


def test_noalloc_gate_matches_mps_apply_gates():
    import torch

    from paper_2303_03681_gb300 import mps

    n, q, chi_max = 10, 4, 32
    rng = make_rng(77)
    ctx = mps.Context(0)
    st = mps.State(ctx, n, None, chi_max=chi_max, precision="fp64")
    st.apply_gates(brickwork_circuit(n, 6, rng))
    B, lam = st.export()
    chi_l, chi_m, chi_r = B[q].shape[0], B[q].shape[2], B[q + 1].shape[2]
    assert chi_l > 1 and chi_r > 1

    dev = torch.device("cuda", 0)
    kmax = min(chi_max, 2 * chi_l, 2 * chi_r)
    bl = torch.zeros(chi_l * 2 * max(chi_m, kmax), dtype=torch.complex128, device=dev)
    br = torch.zeros(max(chi_m, kmax) * 2 * chi_r, dtype=torch.complex128, device=dev)
    bl[: B[q].size] = torch.from_numpy(B[q].reshape(-1)).to(dev)
    br[: B[q + 1].size] = torch.from_numpy(B[q + 1].reshape(-1)).to(dev)
    lam_l = torch.from_numpy(lam[q].copy()).to(dev)
    lam_out = torch.zeros(kmax, dtype=torch.float64, device=dev)
    chi_out = torch.zeros(1, dtype=torch.int32, device=dev)
    fn = _noalloc(mps.library())
    stream = torch.cuda.current_stream().cuda_stream
    ref = orc.MPS([b.copy() for b in B], [x.copy() for x in lam])

    for call in range(2):
        u = haar_su4(rng)
        gl = type(brickwork_circuit(2, 1, rng))(n, np.array([q], np.int32), np.array([2], np.int32), u[None])
        st.apply_gates(gl)
        Bref, lamref = st.export()
        g = np.ascontiguousarray(np.stack([u.real, u.imag], axis=-1).reshape(-1))
        rc = fn(0, ctypes.c_void_p(stream), chi_l, chi_m, chi_r, ctypes.c_void_p(bl.data_ptr()),
                ctypes.c_void_p(br.data_ptr()), ctypes.c_void_p(lam_l.data_ptr()), ctypes.c_void_p(lam_out.data_ptr()),
                g.ctypes.data_as(ctypes.c_void_p), chi_max, 0.0, ctypes.c_void_p(chi_out.data_ptr()))
        assert rc == 0, mps.library().mps_last_error()
        torch.cuda.synchronize()
        k = int(chi_out.item())
        assert k == Bref[q].shape[2]
        assert np.allclose(lam_out[:k].cpu().numpy(), lamref[q + 1], rtol=0, atol=1e-10)
        got_l = bl[: chi_l * 2 * k].cpu().numpy().reshape(chi_l, 2, k)
        got_r = br[: k * 2 * chi_r].cpu().numpy().reshape(k, 2, chi_r)
        theta_got = np.einsum("aim,mjb->aijb", got_l, got_r)
        theta_ref = np.einsum("aim,mjb->aijb", Bref[q], Bref[q + 1])
        assert np.max(np.abs(theta_got - theta_ref)) <= 1e-10
        # the FP64 oracle's Hastings update of the same tensors
        orc.apply_2q(ref, q, u, chi_max, 0.0)
        assert ref.B[q].shape[2] == k
        assert np.allclose(lam_out[:k].cpu().numpy(), ref.lam[q + 1], rtol=0, atol=1e-10)
        theta_orc = np.einsum("aim,mjb->aijb", ref.B[q], ref.B[q + 1])
        assert np.max(np.abs(theta_got - theta_orc)) <= 1e-10
        chi_m = k  # the second call starts from the first call's output


def test_noalloc_rejects_sizes_beyond_the_scratch():
    from paper_2303_03681_gb300 import mps

    fn = _noalloc(mps.library())
    dummy = ctypes.c_void_p(16)
    g = np.zeros(32)
    rc = fn(0, None, 33, 2, 2, dummy, dummy, dummy, dummy, g.ctypes.data_as(ctypes.c_void_p), 8, 0.0, dummy)
    assert rc == mps.MPS_EINVAL
    assert b"1..32" in mps.library().mps_last_error()
    # a device that does not exist is refused before anything is issued
    rc = fn(63, None, 2, 2, 2, dummy, dummy, dummy, dummy, g.ctypes.data_as(ctypes.c_void_p), 8, 0.0, dummy)
    assert rc == mps.MPS_EINVAL
    assert b"no CUDA device 63" in mps.library().mps_last_error()
