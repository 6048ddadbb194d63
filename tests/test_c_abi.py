"""The C ABI from plain C: tests/c_abi/host_calls.c is compiled as C99 with
warnings as errors against include/slu.h, linked against the built library
and run (host entry points only; no GPU needed)."""
import os
import shutil
import subprocess

import pytest

S = pytest.importorskip("paper_2512_04389_b300.slu")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no C compiler")
def test_host_entry_points_from_c(tmp_path):
    exe = tmp_path / "host_calls"
    libdir = os.path.dirname(S.LIB_PATH)
    subprocess.run(
        ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
         "-I", os.path.join(ROOT, "include"),
         os.path.join(ROOT, "tests", "c_abi", "host_calls.c"),
         "-o", str(exe), "-L", libdir, "-l:" + os.path.basename(S.LIB_PATH),
         "-Wl,-rpath," + libdir],
        check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip() == "ok"
