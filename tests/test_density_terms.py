"""The binary64 sweep's exact density sum: the doubled-resolution form equals
the round-each-term form.

The sweep forms each term at twice the fixed-point unit's resolution (mantissa
shifted as a magnitude, sign applied by complement) and recovers the rounding
from the count of odd terms.  ``density_terms_check.c`` restates both forms in
plain C and compares the sums on random, tie-heavy, tiny and signed-zero
inputs at the guard-bit width of every lattice (Q = 5 ... 169).  This checks the
arithmetic identity on the host; the GPU parity tests check the kernel.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_doubled_resolution_terms_equal_rounded_terms(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "density_terms_check")
    src = os.path.join(HERE, "density_terms_check.c")
    subprocess.run([cc, "-O2", "-std=c11", "-o", exe, src, "-lm"], check=True)
    r = subprocess.run([exe, "200000"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    checked = int(r.stdout.split()[1])
    assert checked > 150000, r.stdout
    assert "mismatches 0" in r.stdout
