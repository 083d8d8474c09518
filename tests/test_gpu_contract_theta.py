"""The theta contraction C = Q (B_q B_{q+1}) through mps_contract_theta, against
FP64 on the host (GPU).

Sizes cover a tiny ragged case, one-tile and multi-tile shapes with ragged
64-column tiles and a ragged K, and the full size of the 100-qubit chi = 512
brickwork (2 chi = 1024 rows, chi_m = 512, 1024 columns), where the host
computes 4,000 sampled entries one by one.

Bar: every entry within tol * s_e of the FP64 value, where s_e = sum over the
contraction of |Q||B_q||B_{q+1}| for that entry (the scale of the rounding
error of any summation order).  FP32 CUDA cores and TF32X3 (22-bit pieces)
keep tol = 2e-6 (about 32 units of FP32 rounding: the products round at
2^-24 and the FP32 sums add a few units); BF16X3 keeps 16-bit pieces
(relative 2^-17 per value), tol = 5e-5.
"""

import numpy as np
import pytest

from paper_2303_03681_gb300.inputs import MASTER_SEED, haar_su4, make_rng

pytestmark = pytest.mark.gpu

TOL = {"fp32": 2e-6, "tf32x3": 2e-6, "bf16x3": 5e-5}


def _operands(chi_l, chi_m, chi_r, seed):
    rng = make_rng(seed)
    Bl = (rng.normal(size=(chi_l, 2, chi_m)) + 1j * rng.normal(size=(chi_l, 2, chi_m))) / np.sqrt(2 * chi_m)
    Br = (rng.normal(size=(chi_m, 2, chi_r)) + 1j * rng.normal(size=(chi_m, 2, chi_r))) / np.sqrt(2 * chi_r)
    return Bl.astype(np.complex64), Br.astype(np.complex64), haar_su4(rng)


def _device(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _run(mps, ctx, precision, Bl, Br, u):
    import torch

    chi_l, chi_m, chi_r = Bl.shape[0], Bl.shape[2], Br.shape[2]
    dl, dr = _device(Bl), _device(Br)
    out = torch.full((2 * chi_l, 2 * chi_r), float("nan"), dtype=torch.complex64, device="cuda")
    mps.contract_theta(ctx, precision, chi_l, chi_m, chi_r, dl.data_ptr(), dr.data_ptr(), u, out.data_ptr())
    ctx.synchronize()
    return out.cpu().numpy()


def _entries(Bl, Br, u, rows, cols):
    """FP64 value and error scale of C[(a_l, i), (j, a_r)] for the given (row, col) pairs."""
    chi_r = Br.shape[2]
    Q = u.reshape(2, 2, 2, 2)
    Bl64, Br64 = Bl.astype(np.complex128), Br.astype(np.complex128)
    vals, scales = [], []
    for r, c in zip(rows, cols):
        al, i = divmod(int(r), 2)
        j, ar = divmod(int(c), chi_r)
        v, sc = 0j, 0.0
        for ip in range(2):
            for jp in range(2):
                x, y = Bl64[al, ip, :], Br64[:, jp, ar]
                v += Q[i, j, ip, jp] * np.dot(x, y)
                sc += abs(Q[i, j, ip, jp]) * float(np.dot(np.abs(x), np.abs(y)))
        vals.append(v)
        scales.append(sc)
    return np.array(vals), np.array(scales)


@pytest.fixture(scope="module")
def mps():
    from paper_2303_03681_gb300 import mps as m

    return m


@pytest.fixture(scope="module")
def ctx(mps):
    return mps.Context(0)


@pytest.mark.parametrize("chi_l,chi_m,chi_r", [(1, 1, 1), (3, 5, 7), (64, 64, 64), (100, 37, 200), (130, 96, 33)])
@pytest.mark.parametrize("precision", ["fp32", "tf32x3", "bf16x3"])
def test_contract_theta_small_against_fp64(mps, ctx, precision, chi_l, chi_m, chi_r):
    Bl, Br, u = _operands(chi_l, chi_m, chi_r, MASTER_SEED + 500 + chi_l + chi_m + chi_r)
    got = _run(mps, ctx, precision, Bl, Br, u)
    theta = np.einsum("aim,mjb->aijb", Bl.astype(np.complex128), Br.astype(np.complex128))
    want = np.einsum("ijkl,akld->aijd", u.reshape(2, 2, 2, 2), theta).reshape(2 * chi_l, 2 * chi_r)
    scale = np.einsum("ijkl,akld->aijd", np.abs(u.reshape(2, 2, 2, 2)),
                      np.einsum("aim,mjb->aijb", np.abs(Bl).astype(np.float64), np.abs(Br).astype(np.float64)))
    scale = scale.reshape(2 * chi_l, 2 * chi_r)
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - want) <= TOL[precision] * scale + 1e-30)


@pytest.mark.parametrize("precision", ["fp32", "tf32x3", "bf16x3"])
def test_contract_theta_full_c3_size(mps, ctx, precision):
    chi = 512
    Bl, Br, u = _operands(chi, chi, chi, MASTER_SEED + 510)
    got = _run(mps, ctx, precision, Bl, Br, u)
    assert got.shape == (2 * chi, 2 * chi) and np.all(np.isfinite(got))
    rng = make_rng(MASTER_SEED + 511)
    rows = rng.integers(0, 2 * chi, 4000)
    cols = rng.integers(0, 2 * chi, 4000)
    rows[:4], cols[:4] = [0, 0, 2 * chi - 1, 2 * chi - 1], [0, 2 * chi - 1, 0, 2 * chi - 1]  # the corners
    want, scale = _entries(Bl, Br, u, rows, cols)
    err = np.abs(got[rows, cols] - want)
    print(f"\n{precision} 1024x512x1024: max err / scale = {np.max(err / scale):.3e}")
    assert np.all(err <= TOL[precision] * scale)


def test_contract_theta_rejects_bad_arguments(mps, ctx):
    with pytest.raises(mps.MpsError) as ei:
        mps.contract_theta(ctx, "fp64", 2, 2, 2, 16, 16, np.eye(4), 16)
    assert ei.value.status == mps.MPS_EINVAL
    with pytest.raises(mps.MpsError) as ei:
        mps.contract_theta(ctx, "tf32x3", 0, 2, 2, 16, 16, np.eye(4), 16)
    assert ei.value.status == mps.MPS_EINVAL
