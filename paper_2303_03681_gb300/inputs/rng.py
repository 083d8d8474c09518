"""Seeds for every synthetic workload.

All random draws go through NumPy's PCG64 bit generator so that the oracle
and the CUDA path see bit-identical inputs on any host (x86 or Arm).
"""

import numpy as np

#: Master seed of every synthetic workload (the arXiv number's date, 2023-03-07).
MASTER_SEED = 20230307


def instance_seed(index: int, master: int = MASTER_SEED) -> int:
    """Seed of the ``index``-th instance of a multi-instance workload."""
    return int(master) + int(index)


def make_rng(seed: int) -> np.random.Generator:
    """A fresh PCG64 generator for ``seed``."""
    return np.random.Generator(np.random.PCG64(int(seed)))
