"""include/hylu.h is a C ABI: a C99 program (tests/c_abi_check.c) that
includes only the header compiles with -std=c99 -pedantic -Werror, links
libhylu.so and runs the entry points that need no GPU."""
import os
import shutil
import subprocess

import pytest

from paper_2509_07690_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c99_client_of_the_header(tmp_path):
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    so = build.build()
    libdir = os.path.dirname(so)
    exe = tmp_path / "c_abi_check"
    r = subprocess.run([cc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror",
                        "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c_abi_check.c"),
                        "-o", str(exe), "-L", libdir, "-lhylu", "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "all C ABI checks passed" in run.stdout
