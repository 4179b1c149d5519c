"""The boundary from C: tests/c/abi_smoke.c is compiled as C11 against
include/ahs.h and linked to the engine library (both checked without a GPU); on
a GPU it runs a small lattice through create, init, step, records, measure and
fields, a two-member batch, and the error paths."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2005_14454_gb300")


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    from paper_2005_14454_gb300 import build
    build.build()
    exe = str(tmp_path_factory.mktemp("c") / "abi_smoke")
    cmd = ["gcc", "-std=c11", "-Wall", "-Werror", "-O1", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c", "abi_smoke.c"), "-o", exe,
           os.path.join(PKG, "_ahs.so"), "-Wl,-rpath," + PKG, "-lm"]
    subprocess.check_call(cmd)
    return exe


def test_header_compiles_as_c_and_links(program):
    assert os.access(program, os.X_OK)


@pytest.mark.gpu
def test_c_program_runs_a_lattice(program):
    out = subprocess.run([program], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.count("ok ") == 20
    assert "xi_w" in out.stdout
