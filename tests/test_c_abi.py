"""The library from a program written in plain C (tests/c/chain3_abi.c): the
header compiles as C99 and the shared library links from C.

Without a GPU the program stops before calling the library (exit 3); on the
GPU it runs one timing iteration on the hand-derived chain3 circuit and
checks every result (exit 0).
"""
import os
import subprocess

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _compile(tmp_path):
    lib_dir = os.path.join(ROOT, "paper_2503_11674_b300", "lib")
    if not os.path.exists(os.path.join(lib_dir, "libtdp_b300.so")):
        from paper_2503_11674_b300.build import build
        build()
    exe = str(tmp_path / "chain3_abi")
    cmd = ["gcc", "-std=c99", "-O2", "-Wall", "-Wextra", "-Werror",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
           os.path.join(ROOT, "tests", "c", "chain3_abi.c"), "-o", exe,
           "-L", lib_dir, "-ltdp_b300", "-L", os.path.join(CUDA, "lib64"), "-lcudart", "-lm",
           f"-Wl,-rpath,{lib_dir}", f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_program_compiles_links_and_stops_cleanly(tmp_path):
    exe = _compile(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    expected = 0 if torch.cuda.is_available() else 3
    assert r.returncode == expected, (r.returncode, r.stdout)


@pytest.mark.gpu
def test_c_program_matches_the_hand_derived_circuit(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    exe = _compile(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout
    assert "all results match" in r.stdout
