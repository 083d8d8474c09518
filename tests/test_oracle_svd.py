"""Pins of the oracle's one-sided Jacobi SVD (Algorithm 1) against LAPACK and
the SVD's defining properties (CPU only)."""

import numpy as np
import pytest

from oracle import mps as om
from oracle.svd_jacobi import one_sided_jacobi_svd
from paper_2303_03681_gb300.inputs import brickwork_circuit, make_rng


def _check(A, U, s, Vh):
    scale = np.linalg.norm(A)
    assert np.all(np.diff(s) <= 0)
    assert np.linalg.norm((U * s) @ Vh - A) <= 1e-13 * scale
    assert np.linalg.norm(Vh @ Vh.conj().T - np.eye(Vh.shape[0])) <= 1e-12
    sref = np.linalg.svd(A, compute_uv=False)
    big = sref > 1e-10 * sref[0]
    assert np.allclose(s[: sref.size][big], sref[big], rtol=1e-12, atol=0)


@pytest.mark.parametrize("m,n", [(8, 8), (16, 10), (10, 16), (33, 17), (4, 2)])
def test_jacobi_matches_lapack(m, n):
    rng = make_rng(m * 100 + n)
    A = rng.normal(size=(m, n)) + 1j * rng.normal(size=(m, n))
    _check(A, *one_sided_jacobi_svd(A))


def test_jacobi_rank_deficient_and_graded():
    rng = make_rng(11)
    X = rng.normal(size=(24, 6)) + 1j * rng.normal(size=(24, 6))
    Y = rng.normal(size=(6, 20)) + 1j * rng.normal(size=(6, 20))
    A = X @ Y  # rank 6
    U, s, Vh = one_sided_jacobi_svd(A)
    assert np.all(s[6:] <= 1e-12 * s[0])
    _check(A, U, s, Vh)
    D = np.diag(10.0 ** -np.arange(12))
    Q1, _ = np.linalg.qr(rng.normal(size=(12, 12)) + 1j * rng.normal(size=(12, 12)))
    Q2, _ = np.linalg.qr(rng.normal(size=(12, 12)) + 1j * rng.normal(size=(12, 12)))
    G = Q1 @ D @ Q2
    _, s, _ = one_sided_jacobi_svd(G)
    assert np.allclose(s, np.diag(D), rtol=1e-10, atol=1e-15)


def test_jacobi_rotation_zeroes_the_pair():
    """One rotation makes the two columns orthogonal (the t/tau/c/s formulas)."""
    rng = make_rng(2)
    A = rng.normal(size=(6, 2)) + 1j * rng.normal(size=(6, 2))
    U, s, Vh = one_sided_jacobi_svd(A, max_sweeps=1)
    B = A @ Vh.conj().T
    assert abs(np.vdot(B[:, 0], B[:, 1])) <= 1e-14 * np.linalg.norm(A) ** 2


def test_mps_with_jacobi_svd_matches_lapack_route():
    circ = brickwork_circuit(8, 6, make_rng(4))
    a = om.run_circuit(8, None, circ, chi_max=16)
    b = om.apply_gates(om.product_state(np.zeros(8, int)), circ, 16, 0.0, svd=one_sided_jacobi_svd)
    for la, lb in zip(a.lam, b.lam):
        assert np.allclose(la, lb, rtol=1e-11, atol=1e-13)
    assert om.fidelity(a, b) >= 1 - 1e-12


def _raise_linalg(*args, **kwargs):
    raise np.linalg.LinAlgError("SVD did not converge")


@pytest.mark.parametrize("fail", ["gesdd", "gesdd+gesvd"])
def test_oracle_svd_fallback_matches_lapack_route(monkeypatch, fail):
    """When LAPACK's zgesdd stops with 'SVD did not converge' (it did on an
    aarch64 host), the oracle's gate update falls back to zgesvd and then to
    the Jacobi SVD of Algorithm 1; the truncated MPS is the same."""
    circ = brickwork_circuit(10, 8, make_rng(41))
    ref = om.run_circuit(10, None, circ, chi_max=12, eps_rel=1e-10)
    monkeypatch.setattr(om.np.linalg, "svd", _raise_linalg)
    if fail == "gesdd+gesvd":
        monkeypatch.setattr(om.scipy.linalg, "svd", _raise_linalg)
    got = om.run_circuit(10, None, circ, chi_max=12, eps_rel=1e-10)
    monkeypatch.undo()
    assert ref.bond_dims() == got.bond_dims()
    for la, lb in zip(ref.lam, got.lam):
        assert np.allclose(la, lb, rtol=1e-10, atol=1e-13)
    assert abs(ref.stats.discarded_weight - got.stats.discarded_weight) <= 1e-12
    assert om.fidelity(ref, got) >= 1 - 1e-12
    assert abs(om.canonical_residual(got) - om.canonical_residual(ref)) <= 1e-10
