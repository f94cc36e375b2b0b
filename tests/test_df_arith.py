"""Double-float arithmetic of the FP64-accurate FFT passes (csrc/df.cuh), on
the host: the header's operators compile for the CPU with plain IEEE
binary32 operations, so their error-free and near-exact properties can be
checked against exact rational arithmetic.  Pins: Knuth's two-sum is exact
(s + e = a + b); the double-float sum and product of two normalised pairs are
within 2^-44 of the exact result, relative (the operations' bound is about
2^-46), also when the high parts cancel; results come back normalised
(|lo| <= 2^-24 |hi|); the FP64 -> pair conversion keeps 48 bits.  A dropped error term, a wrong sign or a swapped
operand in any of them fails one of these by orders of magnitude."""
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1709_10010_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include <cstring>
#include <cstdint>
#include "df.cuh"
using pwh::df;
static float f_of(uint32_t u) { float f; std::memcpy(&f, &u, 4); return f; }
static uint32_t u_of(float f) { uint32_t u; std::memcpy(&u, &f, 4); return u; }
int main() {
  char op[8];
  unsigned a, b, c, d;
  while (std::scanf("%7s %x %x %x %x", op, &a, &b, &c, &d) == 5) {
    if (op[0] == 't') {                      // two-sum of two floats
      float s, e;
      pwh::df_two_sum(f_of(a), f_of(b), s, e);
      std::printf("%08x %08x\n", u_of(s), u_of(e));
    } else if (op[0] == 'c') {               // FP64 (bits a:b, high:low) -> pair
      uint64_t bits = ((uint64_t)a << 32) | b;
      double x;
      std::memcpy(&x, &bits, 8);
      df r(x);
      std::printf("%08x %08x\n", u_of(r.hi), u_of(r.lo));
    } else {
      df x(f_of(a), f_of(b)), y(f_of(c), f_of(d));
      df r = op[0] == 'a' ? x + y : (op[0] == 's' ? x - y : x * y);
      std::printf("%08x %08x\n", u_of(r.hi), u_of(r.lo));
    }
  }
  return 0;
}
"""


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    nv = _nvcc()
    if nv is None:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("df")
    src = d / "df_host.cu"
    src.write_text(PROG)
    out = d / "df_host"
    subprocess.run([nv, "-std=c++17", "--expt-relaxed-constexpr", "-O2", "-Xcompiler",
                    "-ffp-contract=off", "-I", CSRC, str(src), "-o", str(out)],
                   check=True, capture_output=True, timeout=300)
    return str(out)


def f32(u):
    return struct.unpack("<f", struct.pack("<I", u))[0]


def bits(f):
    return struct.unpack("<I", struct.pack("<f", f))[0]


def rnd32(x):
    return struct.unpack("<f", struct.pack("<f", x))[0]


def pair(rng):
    """A normalised pair hi + lo: hi a random binary32, lo the binary32
    rounding of a remainder below half an ulp of hi."""
    hi = rnd32(rng.choice([-1, 1]) * rng.uniform(1, 2) * 2.0 ** rng.randint(-20, 20))
    lo = rnd32(hi * rng.uniform(-1, 1) * 2.0 ** -25)
    return hi, lo


def run(exe, lines):
    p = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                       check=True, timeout=60)
    return [tuple(f32(int(t, 16)) for t in l.split()) for l in p.stdout.strip().splitlines()]


def exact(*xs):
    return sum((Fraction(x) for x in xs), Fraction(0))


def test_two_sum_is_exact(exe):
    rng = random.Random(1)
    cases = []
    for _ in range(2000):
        a = rnd32(rng.uniform(-1, 1) * 2.0 ** rng.randint(-30, 30))
        b = rnd32(rng.uniform(-1, 1) * 2.0 ** rng.randint(-30, 30))
        cases.append((a, b))
    out = run(exe, [f"t {bits(a):08x} {bits(b):08x} 0 0" for a, b in cases])
    for (a, b), (s, e) in zip(cases, out):
        assert exact(s, e) == exact(a, b)
        assert s == rnd32(a + b)


@pytest.mark.parametrize("op", ["a", "s", "m"])
def test_sum_difference_product_within_bound(exe, op):
    rng = random.Random({"a": 2, "s": 3, "m": 4}[op])
    cases = []
    for i in range(2000):
        x, y = pair(rng), pair(rng)
        if op != "m" and i % 5 == 0:
            # near cancellation: y close to -x (or x for the difference)
            sgn = -1 if op == "a" else 1
            y = (rnd32(sgn * x[0]), rnd32(sgn * x[1] * rng.uniform(0.5, 1.5)))
        elif op != "m" and i % 5 == 1:
            # the high parts cancel exactly and the low parts differ in scale:
            # the result is the low parts' sum, whose rounding error the
            # accurate addition keeps
            sgn = -1 if op == "a" else 1
            y = (rnd32(sgn * x[0]), rnd32(x[1] * rng.uniform(-1, 1) * 2.0 ** -rng.randint(3, 12)))
        cases.append((x, y))
    lines = [f"{op} {bits(x[0]):08x} {bits(x[1]):08x} {bits(y[0]):08x} {bits(y[1]):08x}"
             for x, y in cases]
    out = run(exe, lines)
    for (x, y), (hi, lo) in zip(cases, out):
        X, Y = exact(*x), exact(*y)
        ref = X * Y if op == "m" else (X + Y if op == "a" else X - Y)
        got = exact(hi, lo)
        assert abs(got - ref) <= Fraction(1, 2 ** 44) * abs(ref), (op, x, y, hi, lo)
        assert abs(lo) <= abs(hi) * 2.0 ** -24
        if ref == 0:
            assert hi == 0 and lo == 0


def test_fp64_to_pair_keeps_48_bits(exe):
    rng = random.Random(5)
    xs = [rng.uniform(-1, 1) * 2.0 ** rng.randint(-40, 40) for _ in range(2000)]
    lines = []
    for x in xs:
        b = struct.unpack("<Q", struct.pack("<d", x))[0]
        lines.append(f"c {b >> 32:08x} {b & 0xffffffff:08x} 0 0")
    out = run(exe, lines)
    for x, (hi, lo) in zip(xs, out):
        assert hi == rnd32(x)
        assert abs(exact(hi, lo) - Fraction(x)) <= Fraction(1, 2 ** 48) * abs(Fraction(x))
