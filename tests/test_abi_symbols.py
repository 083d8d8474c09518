"""The C-ABI library builds, loads and exports every function declared in
include/mps_vqe.h; without a GPU it fails loudly instead of computing on the
CPU (no compute call is made here)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mps_vqe.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2303_03681_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["mps_create", "mps_apply_gates", "mps_energy", "vqe_eval", "mps_hamiltonian_create",
                     "mps_ctx_create", "mps_export", "mps_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_and_reports_version(lib_path):
    from paper_2303_03681_gb300 import mps

    assert "sm_103a" in mps.version()
    assert mps.GATE_DTYPE.itemsize == 264


def test_no_gpu_fails_loudly(lib_path):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2303_03681_gb300 import mps

    with pytest.raises(mps.MpsError):
        mps.Context(0)


def test_input_marshalling_layout():
    import numpy as np

    from paper_2303_03681_gb300 import mps
    from paper_2303_03681_gb300.inputs import brickwork_circuit, make_rng, uccsd_template

    gl = brickwork_circuit(4, 2, make_rng(0))
    arr = mps.gates_to_abi(gl)
    u = arr["u"][0].reshape(16, 2)
    assert np.allclose(u[:, 0] + 1j * u[:, 1], gl.u[0].reshape(-1))
    t = uccsd_template(4, 2)
    ta = mps.template_to_abi(t)
    assert list(ta["param"]) == list(t.param)
    m = ta["m_minus"][0].reshape(16, 2)
    assert np.allclose(m[:, 0] + 1j * m[:, 1], t.m_minus[0].reshape(-1))
