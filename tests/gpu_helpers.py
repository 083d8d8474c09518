"""Helpers shared by the GPU tests (test infrastructure)."""

import numpy as np

from oracle import mps as om


def to_oracle(state):
    """Exported GPU state as an oracle MPS (for fidelity / invariant checks)."""
    B, lam = state.export()
    return om.MPS(B, lam)


def spectra_close(a_lams, b_lams, atol):
    if len(a_lams) != len(b_lams):
        return False
    for x, y in zip(a_lams, b_lams):
        if x.shape != y.shape or not np.allclose(x, y, rtol=0, atol=atol):
            return False
    return True
