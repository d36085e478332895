"""The two-float decision procedure for escapes of 4096 bins or more,
restated in C (tests/native/escape_rule_check.c, the float operations of the
device helpers quant_big and dequant_big), against the double-precision
rules q = rint(fl64(c / w)) and fl32(fl64(q * w)) on inputs crowded at the
rounding boundaries.  The GPU kernels themselves are checked against the
same rules in test_gpu_escape_rule.py."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_two_float_escape_rule_matches_double(tmp_path):
    exe = tmp_path / "escape_rule_check"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math",
                    os.path.join(HERE, "native", "escape_rule_check.c"), "-o", str(exe), "-lm"],
                   check=True)
    out = subprocess.run([str(exe), "400000"], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "mismatches 0" in out.stdout
