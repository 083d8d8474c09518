"""One-sided (Hestenes) Jacobi SVD in FP64 (oracle; test infrastructure only).

Algorithm 1 of the paper ("SVD and one-side jacobi" subsection): sweep over
all column pairs (i, j), i < j; with b_ii = A_i^H A_i, b_jj = A_j^H A_j,
b_ij = A_i^H A_j, rotate the pair when |b_ij| >= eps sqrt(b_ii b_jj) and
accumulate the same rotation into V; stop after a sweep without rotations;
sigma_i = ||A_i||, u_i = A_i / sigma_i; sort by sigma, permuting U and V.

The rotation parameters follow the paper's t / tau / c / s formulas, written
for complex columns: the phase of b_ij is moved onto column j first
(b_ij = |b_ij| e^{i phi}), which makes the pair's Gram matrix real, and the
real rotation zeroes it.  With zeta = (b_jj - b_ii) / (2 |b_ij|):
t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1 / sqrt(1 + t^2), s = t c,
A_i <- c A_i - s e^{-i phi} A_j,   A_j <- s e^{i phi} A_i + c A_j.
"""

import numpy as np


def one_sided_jacobi_svd(A: np.ndarray, eps: float = 1e-15, max_sweeps: int = 60):
    """Returns (U, s, Vh) with A = U diag(s) Vh, s descending; A is m x n, m >= n
    (a wide input is handled through its conjugate transpose)."""
    A = np.array(A, dtype=complex)
    m, n = A.shape
    if m < n:
        U, s, Vh = one_sided_jacobi_svd(A.conj().T, eps, max_sweeps)
        return Vh.conj().T, s, U.conj().T
    V = np.eye(n, dtype=complex)
    tiny = np.finfo(float).tiny
    # columns at the rounding level of A are left alone (a rotation between
    # two of them only reshuffles rounding noise)
    floor = (eps * np.linalg.norm(A)) ** 2
    for _ in range(max_sweeps):
        rotated = False
        for i in range(n - 1):
            for j in range(i + 1, n):
                ai, aj = A[:, i], A[:, j]
                bii = float(np.vdot(ai, ai).real)
                bjj = float(np.vdot(aj, aj).real)
                bij = complex(np.vdot(ai, aj))
                mag = abs(bij)
                if mag <= tiny or mag < eps * np.sqrt(bii * bjj) or min(bii, bjj) <= floor:
                    continue
                rotated = True
                ph = bij / mag
                zeta = (bjj - bii) / (2.0 * mag)
                t = (1.0 if zeta >= 0 else -1.0) / (abs(zeta) + np.sqrt(1.0 + zeta * zeta))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = t * c
                new_i = c * ai - s * np.conj(ph) * aj
                new_j = s * ph * ai + c * aj
                A[:, i], A[:, j] = new_i, new_j
                vi, vj = V[:, i].copy(), V[:, j].copy()
                V[:, i] = c * vi - s * np.conj(ph) * vj
                V[:, j] = s * ph * vi + c * vj
        if not rotated:
            break
    sig = np.linalg.norm(A, axis=0)
    order = np.argsort(-sig, kind="stable")
    sig = sig[order]
    A = A[:, order]
    V = V[:, order]
    U = np.zeros_like(A)
    nz = sig > 0
    U[:, nz] = A[:, nz] / sig[nz]
    return U, sig, V.conj().T
