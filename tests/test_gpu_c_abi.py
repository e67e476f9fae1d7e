"""The C ABI used from a plain C program (gcc, no Python in the process):
tests/c/abi_roundtrip.c is compiled against include/stego.h, linked with
libstego.so and the CUDA runtime, and run."""
import os
import shutil
import subprocess

import pytest

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _cuda_home():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def test_c_program_round_trip(tmp_path):
    need_gpu()  # builds libstego.so
    from paper_0912_0947_gb300 import build as B
    cuda = _cuda_home()
    lib_dir = os.path.dirname(B.LIB)
    exe = str(tmp_path / "abi_roundtrip")
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-Wextra",
           os.path.join(HERE, "c", "abi_roundtrip.c"),
           "-I" + os.path.join(ROOT, "include"), "-I" + os.path.join(cuda, "include"),
           "-L" + lib_dir, "-l:libstego.so", "-Wl,-rpath," + lib_dir,
           "-L" + os.path.join(cuda, "lib64"), "-lcudart", "-Wl,-rpath," + os.path.join(cuda, "lib64"),
           "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "c abi round trip ok" in r.stdout
