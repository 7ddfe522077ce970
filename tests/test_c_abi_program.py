"""The C ABI used by a C program alone (tests/abi_couette.c): compiled with the
system C compiler against include/lbhb.h and the in-tree liblbhb.so.  On a GPU
it must reproduce the exact G = 0 Couette stresses; without one, lb_create must
report a CUDA error through lb_last_error (exit status 3)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1004_5058_gb300")


def build_program(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    import __graft_entry__ as g
    g.build()
    exe = str(tmp_path / "abi_couette")
    src = os.path.join(ROOT, "tests", "abi_couette.c")
    subprocess.run([cc, "-std=c99", "-O2", "-I", os.path.join(ROOT, "include"), src, "-L", PKG, "-llbhb",
                    "-Wl,-rpath," + PKG, "-lm", "-o", exe], check=True)
    return exe


def test_c_program_without_a_device(tmp_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present: the GPU test covers the program")
    r = subprocess.run([build_program(tmp_path)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 3, (r.returncode, r.stdout, r.stderr)
    assert "lb_create" in r.stderr


@pytest.mark.gpu
def test_c_program_couette_stresses(tmp_path):
    r = subprocess.run([build_program(tmp_path)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.strip() == "ok"
