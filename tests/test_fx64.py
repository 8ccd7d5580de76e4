"""The integer-only FP64 arithmetic of the pre-update kernel's row sums
(csrc/fx64.h), checked on the host: the header also compiles as plain C++,
and tests/fx64_check.cpp compares it with references computed other ways."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_fx64_host_check(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path / "fx64_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1711_00121_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "fx64_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    print(out.stdout)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "fx_of ok" in out.stdout and "fx_value ok" in out.stdout and "group sums ok" in out.stdout
