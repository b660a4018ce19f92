"""The device-side tolerance test of the local-moving phase converts exact
128-bit gain sums to double with lv::i128_to_double (csrc/exact.cuh); it
must round exactly as the host compiler does, or a device-controlled run
could stop at another iteration than the host-controlled one.  Checked here
on the CPU (the same header compiled by g++) against the compiler's own
conversion, ties at every rounding position included."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_i128_to_double_rounds_like_the_host_compiler(tmp_path):
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("g++ not available")
    exe = tmp_path / "conv"
    subprocess.check_call([cxx, "-O2", "-I", os.path.join(ROOT, "paper_2501_19004_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "exact_conversion_check.cpp"), "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 mismatches" in r.stdout
