"""The exact-integer helpers of the FP64-accurate tensor-core GEMM on the host.

`csrc/ec_oz_int.h` holds the arithmetic that makes the emulated product exact: the
fixed-point image of each entry against its row's power-of-two scale, the balanced
base-256 digits that become the BF16 slices, the row exponent, and the rounding of the
rebuilt 64-bit integer to binary64 (round to nearest, ties to even).  The header compiles
for host and device; here the host build (`tests/oz_int_check.cpp`, g++) is compared bit for
bit with those definitions written in exact Python integer / rational arithmetic:

* i64_scaled_to_f64_bits(X, sc): the binary64 nearest to X 2^sc (CPython's int -> float
  conversion is correctly rounded, ties to even; ldexp is exact for a normal result);
  refused exactly when the result is not a normal number; the branch-free variant agrees
  wherever it accepts, and accepts every normal result away from the lowest and top
  binades (it tests the exponent before the rounding carry).
* f64_to_fixed64(a, e) = round(a 2^(64 - e)), ties away from zero, for |a| < 2^(e - 1),
  including rows whose largest entry is subnormal.
* row_exponent: |a| < 2^(e - 1), the least such e for a normal a.
* digits8(F): F = sum d_s 256^(7 - s) with |d_s| <= 128, digits of -F = -(digits of F).

No GPU: these run under `-m "not gpu"`.
"""
import math
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2407_11993_gb300", "csrc")


def bits_of(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def val_of(b: int) -> float:
    return struct.unpack("<d", struct.pack("<Q", b))[0]


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("ozint") / "oz_int_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "oz_int_check.cpp"),
                    "-o", exe], check=True, capture_output=True, text=True)

    def run(lines):
        r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                           check=True)
        out = r.stdout.strip().split("\n")
        assert len(out) == len(lines)
        return out
    return run


def ref_scaled(X: int, sc: int):
    """(normal?, bits) of the binary64 nearest to X 2^sc, from the definition."""
    if X == 0:
        return True, 0
    f = float(abs(X))                        # correctly rounded, ties to even
    p = math.frexp(f)[1] - 1                 # leading-one position after rounding
    be = p + 1023 + sc
    if be <= 0 or be >= 2047:
        return False, None
    r = math.ldexp(f, sc)                    # exact: the result is normal
    return True, bits_of(-r if X < 0 else r)


def ref_fixed(a: float, e: int) -> int:
    t = Fraction(a) * Fraction(2) ** (64 - e)
    mag = math.floor(abs(t) + Fraction(1, 2))   # ties away from zero
    return -mag if t < 0 else mag


def ref_row_exponent_ok(a: float, e: int) -> bool:
    if a == 0.0:
        return e == 0
    A = Fraction(abs(a))
    below = A < Fraction(2) ** (e - 1)
    if abs(a) >= 2.0 ** -1022:               # normal: the least such e
        return below and A >= Fraction(2) ** (e - 2)
    return below


def scaled_cases(rng: random.Random):
    cases = []
    for k in range(1, 64):                   # every leading-one position
        for _ in range(6):
            X = rng.getrandbits(k) | (1 << (k - 1))
            if X >= 1 << 63:
                X = (1 << 63) - 1
            cases.append((X if rng.random() < 0.5 else -X, rng.randint(-80, 80)))
    for p in range(53, 63):                  # exact halfway cases, both parities
        sh = p - 52
        for q in ((1 << 52) | 6, (1 << 52) | 7, (1 << 53) - 1):
            X = (q << sh) | (1 << (sh - 1))
            cases += [(X, 0), (-X, -7)]
            cases += [(X + 1, 3), (X - 1, 3)]   # just above / below the tie
    cases += [((1 << 63) - 1, 0), (-((1 << 63) - 1), 5), ((1 << 54) - 1, -40), (1, 0), (-1, 0),
              (0, 12)]
    for _ in range(200):                     # scales reaching subnormal and overflow
        X = rng.getrandbits(rng.randint(1, 63)) or 1
        cases.append((X if rng.random() < 0.5 else -X, rng.randint(-1200, 1100)))
    for p in (0, 40, 62):                    # the normal range's two edges
        for sc in (-1022 - p, -1023 - p, 1023 - p, 1024 - p, 1022 - p):
            cases.append((1 << p, sc))
            cases.append(((1 << (p + 1)) - 1, sc))
    return cases


def test_scaled_integer_to_binary64(checker):
    rng = random.Random(11)
    cases = scaled_cases(rng)
    out = checker([f"S {X} {sc}" for X, sc in cases])
    fast_accepts = 0
    for (X, sc), line in zip(cases, out):
        ok, b, okf, bf = (int(v) for v in line.split())
        rok, rb = ref_scaled(X, sc)
        assert ok == int(rok), (X, sc)
        if rok:
            assert b == rb, (X, sc, hex(b), hex(rb))
        if okf:
            fast_accepts += 1
            assert rok and bf == rb, (X, sc)
        elif X != 0 and rok:
            # the branch-free form tests the exponent before the rounding carry: it may
            # decline only results in the lowest or the top binades
            field = (rb >> 52) & 0x7FF
            assert field <= 1 or field >= 2045, (X, sc)
    assert fast_accepts > len(cases) // 2


def random_double(rng: random.Random, lo: int, hi: int) -> float:
    """A double with a random 52-bit mantissa and binary exponent in [lo, hi]."""
    m = (1 << 52) | rng.getrandbits(52)
    return math.ldexp(m, rng.randint(lo, hi) - 52) * (1 if rng.random() < 0.5 else -1)


def test_fixed_point_image_and_row_exponent(checker):
    rng = random.Random(5)
    vals = [random_double(rng, -1000, 1000) for _ in range(300)]
    vals += [random_double(rng, -30, 30) for _ in range(300)]
    vals += [2.0 ** k for k in (-1022, -1, 0, 1, 52, 1023)] + [-(2.0 ** 0.5), 1.5, -0.75]
    # subnormals, including rows whose largest entry is one
    vals += [val_of(rng.getrandbits(52) | 1) for _ in range(40)] + [val_of(1), val_of((1 << 52) - 1)]
    exps = [int(v) for v in checker([f"E {bits_of(abs(a))}" for a in vals])]
    for a, e in zip(vals, exps):
        assert ref_row_exponent_ok(a, e), (a, e)
    assert int(checker(["E 0"])[0]) == 0
    req, want = [], []
    for a, e in zip(vals, exps):
        for extra in (0, 1, 11, 40, 64, 70):   # a row maximum, and smaller row members
            req.append(f"F {bits_of(a)} {e + extra}")
            want.append(ref_fixed(a, e + extra))
    got = [int(v) for v in checker(req)]
    for r, g, w in zip(req, got, want):
        assert g == w, (r, g, w)
        assert abs(g) < 1 << 63
    # a subnormal row maximum keeps all its bits: F = m 2^11
    m = (1 << 52) - 3
    assert int(checker([f"F {m} -1021"])[0]) == m << 11


def test_balanced_digits(checker):
    rng = random.Random(9)
    Fs = [rng.getrandbits(rng.randint(1, 63)) for _ in range(400)]
    Fs += [0, 1, 127, 128, 129, 255, 256, (1 << 63) - 1, 0x8080808080808080 >> 1,
           sum(128 << (8 * s) for s in range(7))]
    Fs += [-F for F in Fs]
    out = checker([f"D {F}" for F in Fs])
    digits = {}
    for F, line in zip(Fs, out):
        d = [int(v) for v in line.split()]
        assert len(d) == 8 and all(abs(x) <= 128 for x in d), (F, d)
        assert sum(x * 256 ** (7 - s) for s, x in enumerate(d)) == F, (F, d)
        digits[F] = d
    for F in Fs:
        assert digits[-F] == [-x for x in digits[F]]


def test_split_round_trip(checker):
    """fixed point -> digits -> value: within half a unit of 2^(e-64) of the entry, and
    exact for entries without bits below it (the row maximum itself always is)."""
    rng = random.Random(3)
    vals = [random_double(rng, -60, 60) for _ in range(200)]
    exps = [int(v) for v in checker([f"E {bits_of(abs(a))}" for a in vals])]
    emax = max(exps)
    Fs = [int(v) for v in checker([f"F {bits_of(a)} {emax}" for a in vals])]
    ds = checker([f"D {F}" for F in Fs])
    for a, e, F, line in zip(vals, exps, Fs, ds):
        d = [int(v) for v in line.split()]
        back = Fraction(sum(x * 256 ** (7 - s) for s, x in enumerate(d))) * Fraction(2) ** (emax - 64)
        err = abs(back - Fraction(a))
        assert err <= Fraction(2) ** (emax - 65), (a, emax)
        if e == emax:
            assert err == 0, a
