"""The C ABI used from C alone: include/msasm.h compiles as C99 with every warning an error, a client
links against libmsasm.so and the CUDA runtime, and on a GPU it assembles, checks itself and round-trips
the stored tables (tests/c_client/assemble_box.c)."""
import os
import shutil
import subprocess

import pytest

import paper_2107_09568_gb300 as msasm
from paper_2107_09568_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_client", "assemble_box.c")


def _cuda_home():
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _build_client(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    msasm.load()                                   # builds libmsasm.so if it is missing
    lib_dir = os.path.dirname(_lib.library_path())
    cuda = _cuda_home()
    exe = str(tmp_path / "assemble_box")
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(cuda, "include"), SRC, "-o", exe, "-L", lib_dir, "-lmsasm",
           "-L", os.path.join(cuda, "lib64"), "-lcudart", "-lm",
           f"-Wl,-rpath,{lib_dir}", f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_header_is_c99_and_a_c_client_links(tmp_path):
    assert os.path.exists(_build_client(tmp_path))


@pytest.mark.gpu
def test_c_client_assembles_and_round_trips_the_tables(tmp_path):
    exe = _build_client(tmp_path)
    r = subprocess.run([exe, str(tmp_path / "cross_q2.msasm")], capture_output=True, text=True, timeout=600)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("ok")
