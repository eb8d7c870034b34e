"""The C ABI from plain C: include/lbm.h compiles as C (CPU test), and a C
program driving the library steps a square duct to the oracle's flux (GPU
test)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1111_1129_gb300 import build as lib_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi_example.c")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _cc():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    return cc


def _cuda_include():
    inc = os.path.join(CUDA, "include")
    if not os.path.exists(os.path.join(inc, "cuda_runtime_api.h")):
        pytest.skip("CUDA headers not found")
    return inc


def test_header_and_example_compile_as_c(tmp_path):
    obj = tmp_path / "c_abi_example.o"
    res = subprocess.run([_cc(), "-std=c99", "-Wall", "-Wextra", "-Werror", "-c", SRC,
                          "-I", os.path.join(ROOT, "include"), "-I", _cuda_include(),
                          "-o", str(obj)], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr


@pytest.mark.gpu
def test_c_program_matches_the_oracle(tmp_path):
    lib = lib_build.build()
    exe = tmp_path / "c_abi_example"
    libdir = os.path.dirname(lib)
    res = subprocess.run([_cc(), "-std=c99", "-O2", SRC, "-I", os.path.join(ROOT, "include"),
                          "-I", _cuda_include(), "-L", libdir, "-l:" + os.path.basename(lib),
                          "-L", os.path.join(CUDA, "lib64"), "-lcudart",
                          "-Wl,-rpath," + libdir, "-Wl,-rpath," + os.path.join(CUDA, "lib64"),
                          "-o", str(exe)], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    nx, ny, nz, steps = 10, 12, 8, 300
    run = subprocess.run([str(exe), str(nx), str(ny), str(nz), str(steps)],
                         capture_output=True, text=True, timeout=300)
    assert run.returncode == 0, run.stderr
    n, mass, flux = run.stdout.split()
    flags = np.zeros((nz, ny, nx), np.uint8)
    flags[:, 0, :] = flags[:, -1, :] = 1
    flags[:, :, 0] = flags[:, :, -1] = 1
    wp = 1.0 / 0.8
    _, obs, _, _ = oracle.run(flags, 4, wp, oracle.omega_minus(wp), (0.0, 0.0, 1e-5), steps)
    n_ref = int((flags == 0).sum())
    assert int(n) == n_ref
    # stored mass is conserved exactly; the reported sum rounds once per warp
    assert abs(float(mass) - n_ref) <= 1e-12 * n_ref
    flux_ref = obs[-1, 3] / n_ref
    assert abs(float(flux) - flux_ref) <= 1e-11 * abs(flux_ref)
