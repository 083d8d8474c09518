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


C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "mps_vqe.h"

int main(void) {
  mps_ctx* ctx = NULL;
  mps_status rc = mps_ctx_create(0, NULL, &ctx);
  if (rc != MPS_OK) {  /* no usable GPU: a status and a message, no abort */
    printf("status %d: %s\n", (int)rc, mps_last_error());
    return ctx == NULL ? 3 : 1;
  }
  mps_config cfg;
  memset(&cfg, 0, sizeof cfg);
  cfg.chi_max = 4;
  cfg.precision = MPS_PREC_FP64;
  cfg.svd_fp64 = 1;
  mps_state* st = NULL;
  rc = mps_create(ctx, 2, NULL, &cfg, &st);
  mps_gate g;
  memset(&g, 0, sizeof g);
  g.q = 0;
  g.arity = 2;
  for (int k = 0; k < 4; ++k) g.u[2 * (5 * k)] = 1.0;  /* identity */
  if (rc == MPS_OK) rc = mps_apply_gates(st, &g, 1, NULL);
  uint8_t ops[2] = {3, 0};
  double coeff = 1.0, e = 0.0;
  mps_ham* h = NULL;
  if (rc == MPS_OK) rc = mps_hamiltonian_create(ctx, 2, 1, ops, &coeff, &h);
  if (rc == MPS_OK) rc = mps_energy(st, h, &e, NULL);
  printf("status %d energy %.3f\n", (int)rc, e);
  mps_ham_destroy(h);
  mps_destroy(st);
  mps_ctx_destroy(ctx);
  return rc == MPS_OK && e == 1.0 ? 0 : 2;
}
"""


def test_plain_c_client_compiles_links_and_fails_cleanly(lib_path, tmp_path):
    """The header is C99 and the library links from C; without a GPU the
    first call returns a status (MPS_ECUDA) instead of aborting, and with
    one the client applies a gate and reads <Z_0> = 1."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(lib_path)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-o", str(exe), "-L", libdir, "-l:libmpsvqe.so", f"-Wl,-rpath,{libdir}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    import torch

    if torch.cuda.is_available():
        assert run.returncode == 0, run.stdout + run.stderr
    else:
        assert run.returncode == 3 and run.stdout.startswith("status 3:"), run.stdout + run.stderr
