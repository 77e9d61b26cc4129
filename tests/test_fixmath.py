"""The 128-bit integer helpers of the FP64 pair sweep (csrc/fixmath.cuh),
compiled for the host and checked against exact Python integers: squared
distances, binary64 rounding of 128-bit integers, the DSF interval key and
offset from that binary64, and force components rounded once into the
fixed point."""
import os
import random
import struct
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2411_11988_gb300", "csrc", "fixmath.cuh")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include "fixmath.cuh"
int main() {
  char op[8];
  while (scanf("%7s", op) == 1) {
    if (op[0] == 'n') {  // norm2 dx dy dz -> hi lo key x_bits s_bits
      long long dx, dy, dz;
      scanf("%lld %lld %lld", &dx, &dy, &dz);
      fm::u128 r = fm::norm2(dx, dy, dz);
      int p = fm::msb128(r);
      double x = 0.0;
      double s = p >= 0 ? fm::u128_to_dbl(r, p, 96) : 0.0;
      int key = p >= 0 ? fm::dsf_key(s, &x) : -1;
      printf("%llu %llu %d %llu %llu\n", r.hi, r.lo, key, fm::dbl_bits(x), fm::dbl_bits(s));
    } else if (op[0] == 'f') {  // fixf f_bits scale -> result bad
      unsigned fb;
      int sc;
      scanf("%u %d", &fb, &sc);
      float f;
      memcpy(&f, &fb, 4);
      int bad = 0;
      long long r = fm::fixf(f, sc, &bad);
      printf("%lld %d\n", r, bad);
    } else {  // mulfix f_bits d k -> result bad
      unsigned long long fb;
      long long d;
      int k;
      scanf("%llu %lld %d", &fb, &d, &k);
      int bad = 0;
      long long r = fm::mulfix(fm::bits_dbl(fb), d, k, &bad);
      printf("%lld %d\n", r, bad);
    }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    d = tmp_path_factory.mktemp("fixmath")
    src = d / "drv.cpp"
    src.write_text(DRIVER)
    exe = d / "drv"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.dirname(HDR), str(src), "-o", str(exe)],
                   check=True)
    return str(exe)


def _run(exe, lines):
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    return out.stdout.split("\n")


def _dbl(bits):
    return struct.unpack("<d", struct.pack("<Q", bits))[0]


def _bits(v):
    return struct.unpack("<Q", struct.pack("<d", v))[0]


def _round_half_up_dbl(num, scale):
    """binary64 of num * 2^-scale, the 53 leading bits rounded half up."""
    p = num.bit_length() - 1
    if p <= 52:
        m = num << (52 - p)
    else:
        m = ((num >> (p - 53)) + 1) >> 1
        if m >> 53:
            m >>= 1
            p += 1
    return _dbl(((p - scale + 1023) << 52) | (m & ((1 << 52) - 1)))


def test_norm2_key_and_offset(driver):
    rng = random.Random(3)
    cases = [(0, 0, 8), (1, 2, 3), (2 ** 51, 0, 0), (-(2 ** 51) + 5, 2 ** 50 - 3, -(2 ** 49))]
    for _ in range(3000):
        e = rng.randint(20, 52)
        cases.append(tuple(rng.randint(-(2 ** e), 2 ** e) for _ in range(3)))
    out = _run(driver, [f"n {a} {b} {c}" for a, b, c in cases])
    for (a, b, c), line in zip(cases, out):
        hi, lo, key, xb, sb = (int(t) for t in line.split())
        r2 = a * a + b * b + c * c
        assert (hi << 64) | lo == r2
        p = r2.bit_length() - 1
        if r2:
            sv = _dbl(sb)
            assert sv == _round_half_up_dbl(r2, 96)
            # key = top 18 bits of the binary64 s (exponent, 6 mantissa bits)
            assert key == _bits(sv) >> 46
            s0 = _dbl(key << 46)
            x = _dbl(xb)
            # the offset from the interval start is exact
            assert Fraction(x) == Fraction(sv) - Fraction(s0)
            assert 0 <= x < s0 / 64
            if p >= 6:
                # the interval of the exact integer, unless rounding s carried
                # it onto the next interval's start
                k_exact = ((p - 96 + 1023) << 6) | ((r2 >> (p - 6)) & 63)
                assert key == k_exact or (key == k_exact + 1 and x == 0.0)


def _exact_mulfix(f, d, k):
    v = Fraction(f) * d / Fraction(2) ** k
    a = abs(v)
    r = int(a + Fraction(1, 2))  # half away from zero
    return -r if v < 0 else r


def test_mulfix_rounds_once(driver):
    rng = random.Random(5)
    cases = [(0.0, 5, 4), (1.0, 0, 4), (1.5, 3, 1), (-2.5, 7, 2), (3.0, -1, 1)]
    for _ in range(3000):
        f = rng.uniform(-1, 1) * 2.0 ** rng.randint(-30, 12)
        d = rng.randint(-(2 ** 52), 2 ** 52)
        k = rng.randint(4, 11)
        cases.append((f, d, k))
    out = _run(driver, [f"m {_bits(f)} {d} {k}" for f, d, k in cases])
    for (f, d, k), line in zip(cases, out):
        r, bad = (int(t) for t in line.split())
        want = _exact_mulfix(f, d, k)
        if abs(want) >= 2 ** 62:
            assert bad == 1
        else:
            assert bad == 0 and r == want, (f, d, k, r, want)
    # overflow and non-finite inputs are flagged
    out = _run(driver, [f"m {_bits(2.0 ** 40)} {2 ** 52} 4", f"m {_bits(float('inf'))} 3 4"])
    assert [int(t) for t in out[0].split()][1] == 1
    assert [int(t) for t in out[1].split()][1] == 1


def _fbits(v):
    return struct.unpack("<I", struct.pack("<f", v))[0]


def _fval(bits):
    return struct.unpack("<f", struct.pack("<I", bits))[0]


def test_fixf_rounds_once(driver):
    """binary32 to fixed point: round half away from zero of the exact
    product, 0 for subnormals, the flag at 2^62 and for inf/NaN."""
    rng = random.Random(11)
    cases = [(0.0, 44), (-0.0, 44), (1.0, 44), (-1.5, 1), (0.75, 1), (-0.25, 1), (2.0 ** -24, 0),
             (1.5 * 2.0 ** -25, 0), (2.0 ** -25, 0), (1.0e-40, 44)]
    for _ in range(4000):
        f = _fval(_fbits(rng.uniform(-1, 1) * 2.0 ** rng.randint(-60, 30)))
        cases.append((f, rng.choice([39, 44, rng.randint(0, 50)])))
    # exact halves: integers + 1/2 scaled
    for _ in range(500):
        k = rng.randint(0, 2 ** 22)
        sc = rng.randint(1, 20)
        v = (2 * k + 1) / 2.0 ** (sc + 1)
        cases.append((_fval(_fbits(v)) * rng.choice([1, -1]), sc))
    out = _run(driver, [f"f {_fbits(f)} {sc}" for f, sc in cases])
    for (f, sc), line in zip(cases, out):
        r, bad = (int(t) for t in line.split())
        if _fbits(abs(f)) < 0x800000:  # zero or subnormal
            assert (r, bad) == (0, 0)
            continue
        v = Fraction(f) * 2 ** sc
        a = abs(v)
        want = int(a + Fraction(1, 2))
        want = -want if v < 0 else want
        if abs(want) >= 2 ** 62:
            assert bad == 1
        else:
            assert bad == 0 and r == want, (f, sc, r, want)
    out = _run(driver, [f"f {_fbits(2.0 ** 20)} 44", f"f {_fbits(float('inf'))} 4", f"f {0x7FC00000} 4"])
    assert [int(t) for t in out[0].split()][1] == 1
    assert [int(t) for t in out[1].split()][1] == 1
    assert [int(t) for t in out[2].split()][1] == 1
