"""The binary64 sweep's exact density sum: the doubled-resolution form equals
the round-each-term form, and the round-each-term form stays within its
error bound.

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


def _fixed_density(vals, q):
    """The binary64 sweep's density of q values, restated with exact Python
    integers: every value rounded to the unit 2^(emax - 1075 - GB) (emax the
    largest biased exponent, GB = 10 - ceil(log2 q) guard bits; halves away
    from zero), the integer sum converted to binary64 (round to nearest even)
    and scaled by the unit (a power of two, exact)."""
    import math
    from fractions import Fraction
    gb = 10 - (q - 1).bit_length()
    emax = max((math.frexp(abs(v))[1] + 1022) for v in vals if v != 0.0) if any(vals) else 0
    k = emax - 1075 - gb
    unit = Fraction(2) ** k
    acc = 0
    for v in vals:
        t = abs(Fraction(v)) / unit
        r = int(t + Fraction(1, 2))        # floor(|v|/unit + 1/2)
        acc += r if v >= 0 else -r
    return math.ldexp(float(acc), k), unit, emax


def _ulp_of_exponent(e):
    from fractions import Fraction
    return Fraction(2) ** (e - 1075)


@pytest.mark.parametrize("q", [19, 111, 169])
def test_fixed_point_density_error_bound(q):
    """The exact fixed-point density differs from the exact sum of its q
    inputs by at most q/2 units (each term rounded to the unit, unit =
    2^-GB ulp of the largest input) plus half an ulp of the result (the
    final conversion).  Checked on random inputs with exponents spread over
    40 binades, on heavy cancellation (the sum far below the largest input),
    and on ties (inputs that are odd multiples of half a unit).  The same
    cases give the sequential binary64 sum's error for comparison: the bound
    on the fixed-point form is independent of the order of the terms."""
    import math
    import random
    from fractions import Fraction
    rng = random.Random(1504 + q)
    worst_fixed = Fraction(0)
    worst_seq = Fraction(0)
    for case in range(400):
        kind = case % 4
        if kind == 0:      # signs and 40 binades of magnitude
            vals = [rng.choice((-1, 1)) * rng.random() * 2.0 ** -rng.randint(0, 40)
                    for _ in range(q)]
        elif kind == 1:    # cancellation: pairs of near-opposite values
            half = [rng.random() * 2.0 ** -rng.randint(0, 20) for _ in range(q // 2)]
            vals = half + [-h * (1 + 1e-12 * rng.random()) for h in half]
            vals += [rng.random() * 1e-9] * (q - len(vals))
        elif kind == 2:    # population-like: w_i Phi with small deviations
            phi = rng.uniform(-3, 3)
            vals = [phi * rng.random() ** 6 * (1 + 1e-3 * rng.gauss(0, 1)) for _ in range(q)]
        else:              # ties: odd multiples of half the unit of a largest value 1.5
            gb = 10 - (q - 1).bit_length()
            u = 2.0 ** (-52 - gb)
            vals = [1.5] + [rng.choice((-1, 1)) * (2 * rng.randint(0, 2 ** 20) + 1) * u / 2
                            for _ in range(q - 1)]
        rng.shuffle(vals)
        got, unit, emax = _fixed_density(vals, q)
        exact = sum(Fraction(v) for v in vals)
        err = abs(Fraction(got) - exact)
        ulp_res = Fraction(math.ulp(got)) if got != 0.0 else Fraction(0)
        bound = q * unit / 2 + ulp_res / 2
        assert err <= bound, (case, float(err), float(bound))
        seq = 0.0
        for v in vals:
            seq += v
        ulp_max = _ulp_of_exponent(emax)
        worst_fixed = max(worst_fixed, err / ulp_max)
        worst_seq = max(worst_seq, abs(Fraction(seq) - exact) / ulp_max)
    # in ulps of the largest input: the term roundings alone stay below
    # q 2^-(GB+1); the sequential sum is not bounded by anything that small
    gb = 10 - (q - 1).bit_length()
    assert float(worst_fixed) <= q * 2.0 ** -(gb + 1) + 2.0 ** ((q - 1).bit_length() - 1)
    assert worst_seq > 0
