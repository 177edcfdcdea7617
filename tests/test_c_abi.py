"""The boundary is a C ABI: include/bcgpu.h compiles as C11 and a C program
links against libbcgpu.so with no Python in between (tests/c/path_graph.c
checks BC of a weighted path against its closed form)."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "path_graph.c")


def _cc():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    return cc


def test_header_compiles_as_c(tmp_path):
    obj = tmp_path / "path_graph.o"
    subprocess.run([_cc(), "-std=c11", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"), "-c",
                    SRC, "-o", str(obj)], check=True)


@pytest.mark.gpu
def test_c_program_against_the_library(tmp_path):
    import paper_1701_05975_gb300 as bc

    lib = bc.LIB_PATH
    assert os.path.exists(lib), "build the library first"
    exe = tmp_path / "path_graph"
    subprocess.run([_cc(), "-std=c11", "-I", os.path.join(ROOT, "include"), SRC, "-o", str(exe),
                    "-L", os.path.dirname(lib), "-lbcgpu", "-Wl,-rpath," + os.path.dirname(lib), "-lm"], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "ok"
