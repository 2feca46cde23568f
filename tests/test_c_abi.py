"""The C ABI from plain C (CPU): tests/c/abi_host.c compiles with gcc -std=c99 -Wall
-Werror against include/*.h, links against the built library and runs its host-only
calls (error strings, the recoupling coefficient, a plan-only handle)."""
import os
import shutil
import subprocess

import pytest

lib = pytest.importorskip("paper_2407_07411_gb300")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(lib.LIB_PATH)
    exe = tmp_path / "abi_host"
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c", "abi_host.c"), "-o", str(exe), "-L", libdir, "-ldmrg_gb300",
           f"-Wl,-rpath,{libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "c abi ok" in r.stdout, r.stdout + r.stderr
