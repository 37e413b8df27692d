"""Host build of the 128-bit fixed-point sums of the atomic pull gather:
conversions against exact rationals (Python's int / int division rounds
correctly to nearest, ties to even)."""
import ctypes
import math
import os
import random
import struct
import subprocess
import tempfile
from fractions import Fraction

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def fx():
    d = tempfile.mkdtemp(prefix="fx128_")
    so = os.path.join(d, "libfxh.so")
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-shared", "-fPIC",
                    os.path.join(HERE, "fx128_host.cpp"), "-o", so], check=True)
    lib = ctypes.CDLL(so)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    lib.fxh_scale.argtypes = [ctypes.c_int] * 3
    lib.fxh_from_double.argtypes = [ctypes.c_double, ctypes.c_int, u64p, u64p]
    lib.fxh_from_bits.argtypes = [ctypes.c_double, ctypes.c_int, u64p, u64p]
    lib.fxh_to_double.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int]
    lib.fxh_to_double.restype = ctypes.c_double
    lib.fxh_sum.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                            ctypes.POINTER(ctypes.c_int)]
    lib.fxh_sum.restype = ctypes.c_double
    return lib


def bexp(x):
    return (struct.unpack("<Q", struct.pack("<d", x))[0] >> 52) & 0x7FF


def to_double(fx, X, L):
    return fx.fxh_to_double(X & (2**64 - 1), X >> 64, L)


def exact_float(fr):
    """Correctly rounded (nearest, ties to even) double of a non-negative rational."""
    if fr == 0:
        return 0.0
    return fr.numerator / fr.denominator


def test_to_double_rounding(fx):
    rng = random.Random(5)
    cases = []
    for _ in range(4000):
        bits = rng.randint(1, 127)
        X = rng.getrandbits(bits) | (1 << (bits - 1))
        L = rng.randint(-1150, 900)
        cases.append((X, L))
    # exact ties and near-ties at 53 significant bits
    for _ in range(500):
        top = rng.randint(54, 126)
        m = rng.getrandbits(53) | (1 << 52)
        r = top - 53
        half = 1 << (r - 1)
        for X in ((m << r) | half, (m << r) | (half - 1), (m << r) | (half + 1),
                  ((m | 1) << r) | half):
            cases.append((X, rng.randint(-1000, 500)))
    # subnormal and underflowing results, and the boundary to normal
    for X, L in [(1, -1074), (3, -1075), (1, -1075), (1, -1076), ((1 << 53) - 1, -1126),
                 ((1 << 52), -1074), ((1 << 53) - 1, -1075), (1 << 126, -1200), (5, -1076)]:
        cases.append((X, L))
    for X, L in cases:
        want = exact_float(Fraction(X) * Fraction(2) ** L)
        got = to_double(fx, X, L)
        assert got == want, (X, L, got, want)


def test_to_double_ignores_flag_and_zero(fx):
    assert fx.fxh_to_double(0, 1 << 63, -10) == 0.0
    assert fx.fxh_to_double(3, 1 << 63, -1) == 1.5


def test_from_double_exact_and_truncating(fx):
    rng = random.Random(6)
    lo, hi = ctypes.c_uint64(), ctypes.c_uint64()
    for _ in range(3000):
        x = math.ldexp(rng.random() + 0.5, rng.randint(-1070, 1000))
        if rng.random() < 0.05:
            x = math.ldexp(rng.getrandbits(52), -1074)  # subnormal
        L = rng.randint(-1100, 1000)
        fx.fxh_from_double(x, L, ctypes.byref(lo), ctypes.byref(hi))
        X = lo.value | (hi.value << 64)
        q = Fraction(x) / Fraction(2) ** L
        if X >= 2**127 or q >= 2**127:
            continue  # outside the range fx_scale allows
        assert X == math.floor(q), (x, L)
    fx.fxh_from_double(-0.0, 3, ctypes.byref(lo), ctypes.byref(hi))
    assert lo.value == 0 and hi.value == 0


def test_branch_free_conversion_matches(fx):
    """fx_from_bits (no branches, shifts that clamp) gives fx_from_double's
    words for every input: shifts at and around 0, 64 and 128 bits, below
    the scale, subnormals, zeros; and the exact floor wherever it fits."""
    rng = random.Random(7)
    a, b = (ctypes.c_uint64(), ctypes.c_uint64()), (ctypes.c_uint64(), ctypes.c_uint64())
    cases = []
    for sh in list(range(-70, 140)) + [-2000, -129, -128, 200, 1000]:
        for _ in range(4):
            be = rng.randint(1, 2046)
            x = math.ldexp(1.0 + rng.getrandbits(52) / 2**52, be - 1023)
            cases.append((x, (be - 1075) - sh))  # lsb(x) - L = sh
    for _ in range(2000):
        x = math.ldexp(rng.random() + 0.5, rng.randint(-1070, 1000))
        cases.append((x, rng.randint(-1100, 1000)))
    for _ in range(200):
        cases.append((math.ldexp(rng.getrandbits(52), -1074), rng.randint(-1200, -1000)))
    cases += [(0.0, 5), (-0.0, -7), (5e-324, -1074), (5e-324, -1080), (1.0, 0)]
    for x, L in cases:
        fx.fxh_from_double(x, L, ctypes.byref(a[0]), ctypes.byref(a[1]))
        fx.fxh_from_bits(x, L, ctypes.byref(b[0]), ctypes.byref(b[1]))
        assert (a[0].value, a[1].value) == (b[0].value, b[1].value), (x, L)
        X = b[0].value | (b[1].value << 64)
        q = Fraction(x) / Fraction(2) ** L
        if q < 2**127:
            assert X == math.floor(q), (x, L)


@pytest.mark.parametrize("spread", [0, 10, 40, 56, 80, 300])
def test_sum_is_correctly_rounded_when_exact(fx, spread):
    rng = random.Random(spread)
    for trial in range(60):
        n = rng.randint(1, 4096)
        e0 = rng.randint(-900, 600)
        xs = [math.ldexp(rng.random() + 0.5, e0 - rng.randint(0, spread)) for _ in range(n)]
        if trial % 7 == 0:
            xs[rng.randrange(n)] = 0.0
        g = max(1, n.bit_length())
        arr = (ctypes.c_double * n)(*xs)
        L = ctypes.c_int()
        got = fx.fxh_sum(arr, n, g, ctypes.byref(L))
        exact = sum(Fraction(x) for x in xs)
        bmin = min(bexp(x) for x in xs if x)
        lsb = bmin - 1075 if bmin else -1074
        if L.value <= lsb:
            assert got == exact_float(exact)
        else:
            # shares spanning more than the 127-bit window lose their low bits:
            # error below n * 2^L, far under the 1e-12 relative bound
            assert abs(Fraction(got) - exact) <= n * Fraction(2) ** L.value + Fraction(exact_float(exact)) * Fraction(1, 2**52)


def fold(fx, acc, xs):
    n = len(xs)
    arr = (ctypes.c_double * max(n, 1))(*xs)
    seq = ctypes.c_double()
    fx.fxh_fold.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                            ctypes.POINTER(ctypes.c_double)]
    fx.fxh_fold.restype = ctypes.c_double
    got = fx.fxh_fold(acc, arr, n, ctypes.byref(seq))
    return got, seq.value


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


@pytest.mark.parametrize("kind", ["similar", "wide", "growing", "ties", "tiny", "subnormal"])
def test_binade_fold_equals_sequential_fold(fx, kind):
    """The integer fold of the deterministic gather reproduces the plain
    left-to-right FP64 sum bit for bit."""
    rng = random.Random(hash(kind) & 0xFFFF)
    for trial in range(40):
        n = rng.choice([1, 7, 255, 256, 257, 1000, 3000])
        acc = rng.choice([0.0, 0.0, rng.random(), math.ldexp(rng.random(), -30)])
        if kind == "similar":
            xs = [math.ldexp(1 + rng.random(), -20) for _ in range(n)]
        elif kind == "wide":
            xs = [math.ldexp(rng.random(), rng.randint(-80, 5)) for _ in range(n)]
        elif kind == "growing":
            xs = [math.ldexp(rng.random(), -40 + i // 20) for i in range(n)]
        elif kind == "ties":
            # acc on a coarse grid and shares of exactly half its ulp (or
            # odd multiples of it): every add is a tie
            acc = math.ldexp(rng.randint(2**52, 2**53 - 1), -52)
            xs = [math.ldexp(rng.choice([1, 3, 5, 1]), -53) if rng.random() < 0.7
                  else math.ldexp(rng.random(), -60) for _ in range(n)]
        elif kind == "tiny":
            acc = 1.0
            xs = [math.ldexp(rng.random(), rng.randint(-120, -50)) for _ in range(n)]
        else:
            acc = 0.0
            xs = [math.ldexp(rng.getrandbits(52), -1074) for _ in range(n)]
        for i in range(n):
            r = rng.random()
            if r < 0.05:
                xs[i] = 0.0
            elif r < 0.07:
                xs[i] = -0.0
        got, seq = fold(fx, acc, xs)
        assert bits(got) == bits(seq), (kind, trial, got, seq)


@pytest.mark.parametrize("kind", ["hub", "growing", "ties", "wide"])
def test_segmented_fold_equals_sequential_fold(fx, kind):
    """The segment-parallel fold of long lists (predicted binades, composed
    segment steps, element-wise refold where the prediction misses or the
    value leaves the binade) reproduces the sequential FP64 fold bit for
    bit, and refolds only a few segments."""
    fx.fxh_fold_segmented.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                      ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    fx.fxh_fold_segmented.restype = ctypes.c_double
    rng = random.Random(hash(kind) & 0xFFFF)
    for trial in range(12):
        n = rng.choice([257, 4097, 20000, 60000])
        acc = rng.choice([0.0, rng.random() * 1e-6])
        if kind == "hub":
            xs = [math.ldexp(1 + rng.random(), -30) if rng.random() < 0.7 else 0.0
                  for _ in range(n)]
        elif kind == "growing":
            xs = [math.ldexp(rng.random(), -50 + i // 500) for i in range(n)]
        elif kind == "ties":
            acc = 1.0
            xs = [math.ldexp(rng.choice([1, 3]), -53) for _ in range(n)]
        else:
            xs = [math.ldexp(rng.random(), rng.randint(-70, -20)) for _ in range(n)]
        arr = (ctypes.c_double * n)(*xs)
        red = ctypes.c_int()
        got = fx.fxh_fold_segmented(acc, arr, n, ctypes.byref(red))
        seq = acc
        for x in xs:
            seq = seq + x
        assert bits(got) == bits(seq), (kind, trial)
        # refolds happen where the sum enters a new binade (plus a rare
        # missed prediction next to a power of two)
        first = next((x for x in [acc] + xs if x > 0), 0.0)
        crossings = (bexp(seq) - bexp(first) + 1) if first > 0 else 0
        assert red.value <= crossings + 2, (kind, red.value, crossings)
