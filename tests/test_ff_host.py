"""The compensated-FP32 ("float-float") helpers on the host.

`csrc/ec_ff.h` carries FP64 values as unevaluated sums hi + lo of two FP32 numbers for the
kernels that move FP64 work onto the FP32 pipe (the FP32-pair modal products, the
FP32-pair inverse factor of the plain step, the compensated symmetric product of the
tridiagonalisation).  `tests/ff_check.cpp` compiles the header with the host compiler over
a shim that gives the CUDA intrinsics their documented meaning; each helper is compared
with exact rational arithmetic:

* split(a): hi = a truncated to 24 significant bits, lo = the remainder a - hi truncated
  to 24 bits (0 below FP32's normal range), so |a - hi - lo| < 2^-47 |a|.
* split_fast(a): the same hi; lo = the remainder rounded to 24 bits, 0 when |a| < 2^-74.
* add: the high part is the correctly rounded sum of the high parts, and the pair keeps
  the sum to ~2^-46 of the operands.
* madd: the product of two pairs added with the same accuracy, less the dropped al bl.
* a dot product of FP64 vectors cut by split_fast and summed by madd stays within a small
  multiple of 2^-47 sum |a_i b_i| of the exact value (the "about 48 bits" the kernels rely on).

No GPU: these run under `-m "not gpu"`.
"""
import math
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2407_11993_gb300", "csrc")


def b64(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def b32(x: float) -> int:
    return struct.unpack("<I", struct.pack("<f", x))[0]


def f32(b: int) -> float:
    return struct.unpack("<f", struct.pack("<I", b))[0]


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("ff") / "ff_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC,
                    os.path.join(HERE, "ff_check.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)

    def run(lines):
        r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                           check=True)
        out = r.stdout.strip().split("\n")
        assert len(out) == len(lines)
        return [[int(v) for v in ln.split()] for ln in out]
    return run


def trunc24(x: Fraction) -> Fraction:
    """x truncated (toward zero) to 24 significant bits."""
    if x == 0:
        return Fraction(0)
    a = abs(x)
    e = math.floor(math.log2(a))
    while Fraction(2) ** e > a:             # guard the float log2 near powers of two
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    u = Fraction(2) ** (e - 23)
    t = math.floor(a / u) * u
    return t if x > 0 else -t


def rn32(x: Fraction) -> float:
    """x rounded to the nearest binary32 (ties to even); x is a double here."""
    return float(np.float32(float(x)))


def random_pair_doubles(rng, n, lo, hi):
    out = []
    for _ in range(n):
        m = (1 << 52) | rng.getrandbits(52)
        out.append(math.ldexp(m, rng.randint(lo, hi) - 52) * (1 if rng.random() < 0.5 else -1))
    return out


def test_split_definitions(checker):
    rng = random.Random(21)
    vals = random_pair_doubles(rng, 400, -60, 60)
    vals += random_pair_doubles(rng, 100, -120, 120)
    vals += random_pair_doubles(rng, 40, -80, -70)            # around split_fast's 2^-74 edge
    vals += [1.0, -1.0, 0.1, -(2.0 ** 0.5), 2.0 ** -126 * 1.5, 3.0e38, 0.0]
    out = checker([f"P {b64(a)}" for a in vals])
    for a, (hi, lo, hf, lf) in zip(vals, out):
        A = Fraction(a)
        H, L, HF, LF = (Fraction(f32(v)) for v in (hi, lo, hf, lf))
        assert H == trunc24(A) and HF == H, a
        r = A - H                                              # at most 29 bits, exact
        want_lo = trunc24(r)
        if abs(want_lo) < Fraction(2) ** -126:
            want_lo = Fraction(0)
        assert L == want_lo, a
        want_lf = Fraction(rn32(r)) if abs(a) >= 2.0 ** -74 else Fraction(0)
        assert LF == want_lf, a
        if a != 0 and abs(a) >= 2.0 ** -74:
            assert abs(A - H - L) < Fraction(2) ** -47 * abs(A), a
            assert abs(A - HF - LF) <= Fraction(2) ** -48 * abs(A), a
    # out of FP32's range: infinities and NaN in hi, lo = 0
    big, nan = checker([f"P {b64(1e300)}", f"P {b64(float('nan'))}"])
    assert f32(big[0]) == math.inf and big[1] == 0 and f32(big[2]) == math.inf and big[3] == 0
    assert math.isnan(f32(nan[0])) and math.isnan(f32(nan[2]))


def pair(rng, scale):
    """A normalised float pair (h, l): |l| <= ulp(h) / 2."""
    x = rng.uniform(-1.0, 1.0) * scale
    h = rn32(Fraction(x))
    l = rn32(Fraction(x) - Fraction(h))
    return h, l


def test_add_and_madd(checker):
    rng = random.Random(8)
    reqA, reqM, cases = [], [], []
    for _ in range(400):
        s = pair(rng, 10.0 ** rng.uniform(-3, 3))
        b = pair(rng, 10.0 ** rng.uniform(-3, 3))
        a = pair(rng, 10.0 ** rng.uniform(-2, 2))
        cases.append((s, a, b))
        reqA.append(f"A {b32(s[0])} {b32(s[1])} {b32(b[0])} {b32(b[1])}")
        reqM.append(f"M {b32(s[0])} {b32(s[1])} {b32(a[0])} {b32(a[1])} {b32(b[0])} {b32(b[1])}")
    outA, outM = checker(reqA), checker(reqM)
    eps = Fraction(2) ** -45
    for (s, a, b), (th, tl), (mh, ml) in zip(cases, outA, outM):
        S, Bv = Fraction(s[0]) + Fraction(s[1]), Fraction(b[0]) + Fraction(b[1])
        # add: high part correctly rounded, pair accurate to ~2^-46 of the operands
        assert f32(th) == rn32(Fraction(s[0]) + Fraction(b[0]))
        got = Fraction(f32(th)) + Fraction(f32(tl))
        assert abs(got - (S + Bv)) <= eps * (abs(Fraction(s[0])) + abs(Fraction(b[0]))), (s, b)
        # madd: (ah + al)(bh + bl) added, al bl dropped
        P = (Fraction(a[0]) + Fraction(a[1])) * Bv
        got = Fraction(f32(mh)) + Fraction(f32(ml))
        bound = eps * (abs(Fraction(s[0])) + abs(Fraction(a[0]) * Fraction(b[0]))) + \
            abs(Fraction(a[1]) * Fraction(b[1]))
        assert abs(got - (S + P)) <= bound, (s, a, b)


@pytest.mark.parametrize("n", [1, 7, 100, 1000])
def test_compensated_dot_product(checker, n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal(n) * np.exp(rng.uniform(-3, 3, n))
    b = rng.standard_normal(n)
    line = "X %d " % n + " ".join(f"{b64(float(x))} {b64(float(y))}" for x, y in zip(a, b))
    (sh, sl), = checker([line])
    got = Fraction(f32(sh)) + Fraction(f32(sl))
    exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))
    scale = sum(abs(Fraction(float(x)) * Fraction(float(y))) for x, y in zip(a, b))
    rel = float(abs(got - exact) / scale)
    print(f"n={n}: |error| / sum|a b| = {rel:.2e}")
    # input cuts 2 x 2^-48, dropped al bl 2^-48, two rounded FMAs 2 x 2^-48 per term, and
    # the low part's own rounding growing with n: (8 + n) 2^-48 covers random data
    assert rel <= (8 + n) * 2.0 ** -48
    # and a plain FP32 dot product would be ~2^-24: the pair form gains ~20 bits or more
    assert rel < 2.0 ** -40
