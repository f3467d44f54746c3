"""CPU check of the host logic that turns the library's device status words
(a tensor-core layer that gave up a bounded wait records it there) into a
status: read, report once, clear; read or clear failures are CUDA errors.
The logic lives in a CUDA-free header (csrc/flags.h); a small C++ program
drives it with a host word standing in for the device symbol."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_take_flag_read_report_clear(tmp_path):
    exe = tmp_path / "flag_logic_check"
    src = os.path.join(ROOT, "tests", "native", "flag_logic_check.cpp")
    inc = os.path.join(ROOT, "paper_1712_00143_gb300", "csrc")
    subprocess.run(["g++", "-std=c++17", "-O1", "-I" + inc, src, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
