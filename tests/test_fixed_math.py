"""Host check of the integer arithmetic of the fixed-point patch apply
(`csrc/fx_math.h`, used by the CUDA kernels of k_patch_fixed.cu) against
exact rational arithmetic (Python's Fraction): scaling a double by 2^k and
rounding to the nearest integer with ties to even, the binary exponent of a
double (as frexp), the split into two 29-bit limbs, and the double nearest to
an exact 128-bit limb sum times 2^e.  Random cases over the whole exponent
range, subnormals, zeros and exact ties."""
import math
import os
import random
import shutil
import subprocess
from fractions import Fraction

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2202_07381_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("fx") / "fixed_math_driver")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, "-o", exe,
                    os.path.join(HERE, "fixed_math_driver.cpp")], check=True)
    return exe


def run(exe, mode, lines):
    out = subprocess.run([exe, mode], input="\n".join(lines) + "\n", capture_output=True,
                         text=True, check=True).stdout.split("\n")
    return [o for o in out if o]


def rne(fr):
    """Nearest integer to a Fraction, ties to even."""
    f = math.floor(fr)
    r = fr - f
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and f % 2 == 1):
        f += 1
    return f


def nearest_double(fr):
    """The double nearest to a Fraction, ties to even (normal range)."""
    if fr == 0:
        return 0.0
    neg, a = fr < 0, abs(fr)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    d = math.ldexp(rne(a / Fraction(2) ** (e - 52)), e - 52)
    return -d if neg else d


def test_scale_round_matches_exact_rounding(driver):
    rng = random.Random(11)
    cases = []
    for _ in range(20000):
        x = rng.choice([-1, 1]) * rng.random() * 2.0 ** rng.randint(-1060, 60)
        u = rng.random()
        if u < 0.03:
            x = 0.0
        elif u < 0.08:
            x = rng.choice([-1, 1]) * 5e-324 * rng.randint(1, 2 ** 40)   # subnormal
        elif u < 0.13:
            x = rng.choice([-1, 1]) * (rng.randint(0, 2 ** 20) + 0.5)    # an exact tie at k = 0
        F = math.frexp(abs(x))[1] if x else 0
        k = 0 if 0.08 <= u < 0.13 else rng.randint(58 - F - 80, 62 - F)
        cases.append((x, k))
    got = run(driver, "s", [f"{x.hex()} {k}" for x, k in cases])
    assert len(got) == len(cases)
    bad = [(x, k, g) for (x, k), g in zip(cases, got) if int(g) != rne(Fraction(x) * Fraction(2) ** k)]
    assert not bad, bad[:3]


def test_exponent_matches_frexp(driver):
    rng = random.Random(12)
    ys = [abs(rng.random() * 2.0 ** rng.randint(-1070, 1020)) or 1.0 for _ in range(5000)]
    ys += [5e-324 * rng.randint(1, 2 ** 52 - 1) for _ in range(500)] + [5e-324, 2.0 ** -1022, 1.0]
    got = run(driver, "e", [y.hex() for y in ys])
    assert [int(g) for g in got] == [math.frexp(y)[1] for y in ys]


def test_split29_recombines_within_the_limb_ranges(driver):
    rng = random.Random(13)
    qs = [rng.randint(-2 ** 58, 2 ** 58) for _ in range(5000)] + [2 ** 58, -2 ** 58, 0, 1, -1,
                                                                  2 ** 28, -2 ** 28, 2 ** 28 - 1]
    got = run(driver, "p", [str(q) for q in qs])
    for q, g in zip(qs, got):
        hi, lo = map(int, g.split())
        assert hi * 2 ** 29 + lo == q and -2 ** 28 <= lo < 2 ** 28 and abs(hi) <= 2 ** 29


def test_round_is_the_nearest_double(driver):
    rng = random.Random(14)
    cases = []
    for _ in range(10000):
        a = [rng.randint(-2 ** 62, 2 ** 62) for _ in range(4)]
        for i in range(rng.randint(0, 3)):
            a[rng.randrange(4)] = 0
        if rng.random() < 0.05:       # a tie: t = (2^53 + 1) 2^10 rounds to even
            a = [0, 0, 0, (2 ** 53 + 1) * 2 ** 10]
        cases.append((a, rng.randint(-900, 800)))
    # |t| above 2^64: an exact half rounds to even, a half plus the lowest bit
    # (only the sticky bit sees it) rounds up
    for t in (2 ** 70 + 2 ** 17, 2 ** 70 + 2 ** 17 + 1, -(2 ** 100 + 2 ** 47), -(2 ** 100 + 2 ** 47 + 1),
              2 ** 70 + 3 * 2 ** 17, 2 ** 118 - 1):
        a0, rest = divmod(t, 2 ** 58)
        cases.append(([a0, 0, 0, rest], 0))
    got = run(driver, "r", [" ".join(map(str, a)) + f" {e}" for a, e in cases])
    assert len(got) == len(cases)
    for (a, e), g in zip(cases, got):
        t = a[0] * 2 ** 58 + (a[1] + a[2]) * 2 ** 29 + a[3]
        ref = nearest_double(Fraction(t) * Fraction(2) ** e)
        assert float.fromhex(g) == ref, (a, e, g, ref)


def nearest_double_any(fr):
    """The double nearest to a Fraction, ties to even, subnormals included:
    below 2^-1022 the grid is the multiples of 2^-1074."""
    if fr == 0:
        return 0.0
    neg, a = fr < 0, abs(fr)
    if a >= Fraction(2) ** -1022:
        return nearest_double(fr)
    d = math.ldexp(rne(a / Fraction(2) ** -1074), -1074)
    return -d if neg else d


def test_round_below_the_normal_range_rounds_once(driver):
    """Results below 2^-1022 must be rounded once, straight to the subnormal
    spacing: rounding first to 53 bits and then again to the subnormal
    precision gets the halfway cases wrong (double rounding)."""
    rng = random.Random(15)
    cases = []
    for _ in range(6000):
        a = [rng.randint(-2 ** 62, 2 ** 62) for _ in range(4)]
        for i in range(rng.randint(0, 3)):
            a[rng.randrange(4)] = 0
        t = a[0] * 2 ** 58 + (a[1] + a[2]) * 2 ** 29 + a[3]
        if t == 0:
            continue
        # put |t 2^e| between 2^-1140 and 2^-1020
        e = rng.randint(-1140, -1020) - (abs(t).bit_length() - 1)
        cases.append((a, e))
    # double-rounding traps: t 2^e = (2k + 1) 2^-1075 + a tiny excess that a
    # first rounding to 53 bits drops (for k >= 2^52 / 2^11 ...) or keeps
    for k in (1, 3, 2 ** 40 + 1, 2 ** 51 - 1, 2 ** 52 - 1):
        for excess in (1, -1, 0):
            t = ((2 * k + 1) << 10) + excess          # (2k+1) 2^10 (+-1), e = -1085
            a0, rest = divmod(t, 2 ** 58)
            cases.append(([a0, 0, 0, rest], -1085))
            cases.append(([-a0, 0, 0, -rest], -1085))   # the negative of it
    got = run(driver, "r", [" ".join(map(str, a)) + f" {e}" for a, e in cases])
    assert len(got) == len(cases)
    for (a, e), g in zip(cases, got):
        t = a[0] * 2 ** 58 + (a[1] + a[2]) * 2 ** 29 + a[3]
        ref = nearest_double_any(Fraction(t) * Fraction(2) ** e)
        assert float.fromhex(g) == ref, (a, e, g, ref)
