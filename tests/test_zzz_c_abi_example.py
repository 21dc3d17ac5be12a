"""The ABI from plain C (tests/c_abi/circle_solve.c): the example compiles as
C11 with warnings as errors against include/bem.h alone and links against the
built library.  Without a GPU it must fail loudly at bem_plan (no host
fallback); on a GPU it solves a Dirichlet problem on a circle and checks the
solution against the unsplit equation (exit status 0)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi", "circle_solve.c")


def _compile(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    from paper_1809_00845_gb300 import bem, build
    build.build()
    libdir = os.path.dirname(bem.LIB_PATH)
    exe = str(tmp_path / "circle_solve")
    cmd = [gcc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-O2", "-I", os.path.join(ROOT, "include"),
           SRC, "-o", exe, "-L", libdir, "-lbem_gb300", "-lm", f"-Wl,-rpath,{libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except ImportError:
        return False


def test_c_example_compiles_links_and_fails_loudly_without_a_gpu(tmp_path):
    exe = _compile(tmp_path)
    if _has_gpu():
        pytest.skip("a CUDA device is present (the GPU test runs the example)")
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 1 and "bem_plan" in r.stderr, (r.returncode, r.stdout, r.stderr)


@pytest.mark.gpu
def test_c_example_solves_on_the_gpu(tmp_path):
    if not _has_gpu():
        pytest.skip("no CUDA device")
    exe = _compile(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
