"""GB300-native MPS circuit simulation and Pauli-sum energy (arXiv:2303.03681).

``paper_2303_03681_gb300.mps`` is the Python binding of the C-ABI library
``libmpsvqe.so`` (CUDA kernels for sm_103a); ``paper_2303_03681_gb300.inputs``
generates seeded synthetic circuits and Hamiltonians.  The CUDA library is
loaded on first use of the binding, never by importing the package.
"""

__version__ = "0.1.0"
