"""Cross-product SVD against the one-sided Jacobi of Algorithm 1 (CPU; the
accuracy half of the SVD study, Results, "Speedup and Scaling").

The paper rejects the cross-product SVD (eigenvectors of A^H A) because
forming A^H A squares the condition number.  In the MPS update this shows
up as follows.  The cross-product returns the singular values at rounding
level as sqrt(u) s_1 ~ 1e-8 s_1 instead of ~1e-16 s_1.  With a truncation
threshold at or below that level, those noise directions are kept, and the
new site tensor C V^H / ||s|| is no longer right-canonical (Eq.
rightcanonicalcondition).  Algorithm 1 keeps the state canonical to
rounding at any threshold.  The energy does not show the damage at this
size, since Eq. expec2 weights the noise directions by lam^2 ~ 1e-16.
"""

import numpy as np
import pytest

from oracle import dense as od
from oracle import mps as om
from oracle.svd_jacobi import one_sided_jacobi_svd
from paper_2303_03681_gb300.inputs import (MASTER_SEED, hf_bits, jw_molecular_hamiltonian, make_rng,
                                           random_integrals, uccsd_template)


def cross_product_svd(A):
    """SVD from the eigen-decomposition of A^H A (the rejected alternative)."""
    w, V = np.linalg.eigh(A.conj().T @ A)
    w, V = w[::-1], V[:, ::-1]
    s = np.sqrt(np.maximum(w, 0.0))
    return A @ V / np.where(s > 0, s, 1.0), s, V.conj().T


@pytest.fixture(scope="module")
def case():
    h, g = random_integrals(4, make_rng(MASTER_SEED + 204))
    ham = jw_molecular_hamiltonian(h, g)
    tmpl, bits = uccsd_template(8, 4), hf_bits(8, 4)
    gates = tmpl.bind(make_rng(5).uniform(-0.3, 0.3, tmpl.n_params))
    return ham, gates, bits, od.energy(od.run(8, bits, gates), ham)


def test_rank_deficient_spectrum():
    rng = make_rng(MASTER_SEED + 205)
    X = rng.normal(size=(32, 6)) + 1j * rng.normal(size=(32, 6))
    Y = rng.normal(size=(6, 24)) + 1j * rng.normal(size=(6, 24))
    A = X @ Y  # rank 6
    s_j = one_sided_jacobi_svd(A)[1]
    s_x = cross_product_svd(A)[1]
    assert np.max(s_j[6:]) <= 1e-14 * s_j[0]
    assert np.max(s_x[6:]) >= 1e-10 * s_x[0]  # sqrt of rounding-level eigenvalues


@pytest.mark.parametrize("eps_rel,broken", [(1e-8, True), (1e-6, False)])
def test_cross_product_breaks_the_canonical_form(case, eps_rel, broken):
    ham, gates, bits, e_exact = case
    jac = om.apply_gates(om.product_state(bits), gates, 16, eps_rel, svd=one_sided_jacobi_svd)
    xp = om.apply_gates(om.product_state(bits), gates, 16, eps_rel, svd=cross_product_svd)
    assert om.canonical_residual(jac) <= 1e-12
    assert (om.canonical_residual(xp) > 0.1) == broken
    for m in (jac, xp):
        assert abs(om.energy(m, ham) - e_exact) <= 1e-10
