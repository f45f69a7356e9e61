"""Host checks of the kernels' exact-arithmetic helpers against rational arithmetic (no GPU).

The exact-integer matvec (Sec. 3.2, the Toeplitz product c T v_k) rests on steps that must be exact or correctly
rounded: Garner's CRT of the four residues, the rounding of the reconstructed integer times a power of two to
FP64, the exact FP32 -> FP64 widening, and the BDF2 band of C (Eq. 1.7); the mixed Arnoldi basis rests on the
FP64 -> float-float split.  Their device code is plain integer and
floating-point C++, so this test compiles the same source text for the host (the few CUDA intrinsics they use
are given host definitions) and compares every result with Python's exact Fraction arithmetic, which rounds
to nearest even like the FP64 conversion it stands in for.
"""
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2003_07020_gb300", "csrc")

SHIMS = r"""
#include <cstdint>
#include <cstring>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#define __device__
#define __forceinline__ inline
#define __restrict__
#define __noinline__ __attribute__((noinline))
struct uint2 { uint32_t x, y; };
struct float2 { float x, y; };
static inline float __double2float_rn(double x) { return (float)x; }
static inline float __uint_as_float(unsigned u) { float f; memcpy(&f, &u, 4); return f; }
static inline int __clz(int x) { return x ? __builtin_clz((unsigned)x) : 32; }
static inline int __clzll(unsigned long long x) { return x ? __builtin_clzll(x) : 64; }
static inline uint32_t __umulhi(uint32_t a, uint32_t b) { return (uint32_t)(((uint64_t)a * b) >> 32); }
static inline uint64_t __umul64hi(uint64_t a, uint64_t b) { return (uint64_t)(((unsigned __int128)a * b) >> 64); }
static inline double __ull2double_rn(unsigned long long x) { return (double)x; }
static inline double __longlong_as_double(long long x) { double d; memcpy(&d, &x, 8); return d; }
static inline long long __double_as_longlong(double x) { long long d; memcpy(&d, &x, 8); return d; }
static inline unsigned __float_as_uint(float f) { unsigned u; memcpy(&u, &f, 4); return u; }
static inline double __hiloint2double(int hi, int lo) {
  return __longlong_as_double((long long)(((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo));
}
template <class T> static inline T __ldg(const T* p) { return *p; }
using std::fma;
using std::ldexp;
"""

MAIN = r"""
int main(int argc, char** argv) {
  const int mode = atoi(argv[1]);
  if (mode == 0) {  // r0 r1 r2 r3 E -> crt_to_double(crt4_top(r, c), E); the 12 Garner words come first
    uint2 c[6];
    for (int i = 0; i < 6; ++i) if (scanf("%u %u", &c[i].x, &c[i].y) != 2) return 1;
    unsigned r[4]; int E;
    while (scanf("%u %u %u %u %d", &r[0], &r[1], &r[2], &r[3], &E) == 5) {
      const uint32_t rq[NP] = {r[0], r[1], r[2], r[3]};
      printf("%016llx\n", (unsigned long long)__double_as_longlong(crt_to_double(crt4_top(rq, c), E)));
    }
  } else if (mode == 1) {  // FP32 bits, d -> f2d_exact
    unsigned u; int d;
    while (scanf("%x %d", &u, &d) == 2) {
      float f; memcpy(&f, &u, 4);
      printf("%016llx\n", (unsigned long long)__double_as_longlong(f2d_exact(f, d)));
    }
  } else if (mode == 3) {  // FP64 bits -> ff_split hi, lo as FP32 bits
    unsigned long long u;
    while (scanf("%llx", &u) == 1) {
      const float2 s = ff_split(__longlong_as_double((long long)u));
      printf("%08x %08x\n", __float_as_uint(s.x), __float_as_uint(s.y));
    }
  } else {  // v_{k-2} v_{k-1} v_k as FP32 bits, k -> band of FP32 rows and of the same values as FP64 rows
    unsigned a, b, cc; int k;
    while (scanf("%x %x %x %d", &a, &b, &cc, &k) == 4) {
      float fv[3]; memcpy(&fv[0], &a, 4); memcpy(&fv[1], &b, 4); memcpy(&fv[2], &cc, 4);
      const double dv[3] = {(double)fv[0], (double)fv[1], (double)fv[2]};
      printf("%016llx %016llx\n", (unsigned long long)__double_as_longlong(bdf_band(&fv[2], 1, k)),
             (unsigned long long)__double_as_longlong(bdf_band(&dv[2], 1, k)));
    }
  }
  return 0;
}
"""


def _between(text, start, end):
    i = text.index(start)
    return text[i:text.index(end, i)]


def _source():
    ntt = open(os.path.join(CSRC, "ntt.cu")).read()
    common = open(os.path.join(CSRC, "common.cuh")).read()
    kern = open(os.path.join(CSRC, "kernels.h")).read()
    ff = open(os.path.join(CSRC, "ff.cuh")).read()
    primes = _between(kern, "constexpr int kNttPrimes", "constexpr uint32_t kNttGen")
    parts = [
        SHIMS, primes, "constexpr int NP = kNttPrimes;\n",
        _between(ntt, "template <int Q> struct Prime", "__device__ __forceinline__ int pad32"),
        _between(common, "__device__ __forceinline__ double f2d_exact", "// Copies the quarter"),
        _between(ntt, "template <int B> __device__ __forceinline__ uint32_t gstep", "// Chunks per row"),
        _between(ff, "__device__ __forceinline__ float2 ff_from_double(double x)", "__device__ __forceinline__ float2 ff_mul"),
        MAIN,
    ]
    return "\n".join(parts), [int(x) for x in primes.split("{")[1].split("}")[0].replace("u", "").split(",")]


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src, primes = _source()
    d = tmp_path_factory.mktemp("exact_helpers")
    cpp, exe = d / "h.cpp", d / "h"
    cpp.write_text(src)
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-o", str(exe), str(cpp)], check=True)
    return str(exe), primes


def _run(exe, mode, lines):
    out = subprocess.run([exe, str(mode)], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    return out.stdout.split("\n")


def _f64(hexbits):
    return struct.unpack("<d", bytes.fromhex(hexbits)[::-1])[0]


def _f32(u):
    return struct.unpack("<f", struct.pack("<I", u))[0]


def _round(v):
    """The FP64 value nearest to the rational v (ties to even), with overflow to infinity."""
    try:
        return float(v)
    except OverflowError:
        return float("inf") if v > 0 else float("-inf")


def test_crt_reconstruction_and_rounding_are_exact(harness):
    exe, primes = harness
    P = 1
    for p in primes:
        P *= p
    garner = []
    for a in range(3):
        for b in range(a + 1, 4):
            c = pow(primes[a], -1, primes[b])
            garner.append("%d %d" % (c, (c << 32) // primes[b]))
    rng = random.Random(7)
    bound = 1 << 117  # |Y| < 2^117 (1 + 2^-45) for the quantised stencil and rows
    ys = [0, 1, -1, 2, -2, bound - 1, -(bound - 1), (1 << 53) + 1, -((1 << 53) + 1), (1 << 64) + 3]
    for _ in range(6000):
        bits = rng.choice([rng.randint(1, 117), 117, 64, 53, 54, 128 - 11])
        bits = min(bits, 117)
        ys.append(rng.choice([1, -1]) * rng.getrandbits(bits))
        # near ties of the 53-bit rounding: a 1 just below the kept bits and nothing after it
        m = rng.getrandbits(53) | (1 << 52)
        s = rng.randint(1, 117 - 54)
        ys.append(rng.choice([1, -1]) * ((m << s) | (1 << (s - 1))))
    lines, cases = list(garner), []
    for y in ys:
        E = rng.choice([0, rng.randint(-250, 100), rng.randint(-1200, -1000), rng.randint(900, 1000)])
        lines.append("%d %d %d %d %d" % tuple([y % p for p in primes] + [E]))
        cases.append((y, E))
    out = _run(exe, 0, lines)
    bad = []
    for (y, E), o in zip(cases, out):
        got = _f64(o)
        want = _round(Fraction(y) * Fraction(2) ** E)
        if got == want:
            continue
        # results below the normal range take the conversion and ldexp: one rounding more is allowed there
        if want != 0 and abs(want) < 2.2250738585072014e-308 and abs(got - want) <= 5e-324:
            continue
        bad.append((y, E, got, want))
    assert not bad, bad[:5]


def test_fp32_widening_is_exact_for_every_class(harness):
    exe, _ = harness
    rng = random.Random(11)
    cases = [(0, 0), (0x80000000, 1), (1, 0), (1, -1), (0x7FFFFF, 1), (0x00800000, -1), (0x7F7FFFFF, 1),
             (0x7F800000, 0), (0xFF800000, -1), (0x7FC00000, 0), (0x7F800001, 1)]
    for _ in range(20000):
        r = rng.random()
        if r < 0.3:
            u = rng.getrandbits(23) | (rng.getrandbits(1) << 31)  # zero and subnormal
        elif r < 0.35:
            u = 0x7F800000 | rng.getrandbits(23) | (rng.getrandbits(1) << 31)  # infinities and NaNs
        else:
            u = rng.getrandbits(32)
        cases.append((u, rng.choice([-1, 0, 1])))
    out = _run(exe, 1, ["%x %d" % c for c in cases])
    for (u, d), o in zip(cases, out):
        f, got = _f32(u), _f64(o)
        if f != f:
            assert got != got, hex(u)
        elif f in (float("inf"), float("-inf")):
            assert got == f, hex(u)
        elif f == 0.0:
            assert got == 0.0 and (o[0] in "89abcdef") == bool(u >> 31), hex(u)
        else:
            assert got == f * 2.0 ** d, (hex(u), d, got)


def test_bdf2_band_matches_eq_1_7(harness):
    # row 0 (BDF1 start): v_0; row 1: 3/2 v_1 - 2 v_0; rows k >= 2: 3/2 v_k - 2 v_{k-1} + 1/2 v_{k-2}; at most
    # two roundings of FP64 arithmetic, so within 2^-51 of the sum of the terms' magnitudes; rows 0 and 1 need
    # one rounding and agree between FP32 and FP64 storage
    exe, _ = harness
    rng = random.Random(13)
    cases = []
    for _ in range(20000):
        vals = []
        for _ in range(3):
            r = rng.random()
            if r < 0.05:
                x = 0.0
            elif r < 0.08:
                x = rng.choice([1, -1]) * 1e-40 * rng.random()
            else:
                x = rng.gauss(0, 1) * 2.0 ** rng.randint(-120, 120)
            vals.append(struct.unpack("<I", struct.pack("<f", x))[0])
        cases.append((vals, rng.randint(0, 3)))
    out = _run(exe, 2, ["%x %x %x %d" % (v[0], v[1], v[2], k) for v, k in cases])
    for (v, k), o in zip(cases, out):
        a2, a1, a0 = [Fraction(_f32(u)) for u in v]  # v_{k-2}, v_{k-1}, v_k
        if k == 0:
            exact, scale = a0, abs(a0)
        elif k == 1:
            exact, scale = Fraction(3, 2) * a0 - 2 * a1, Fraction(3, 2) * abs(a0) + 2 * abs(a1)
        else:
            exact = Fraction(3, 2) * a0 - 2 * a1 + a2 / 2
            scale = Fraction(3, 2) * abs(a0) + 2 * abs(a1) + abs(a2) / 2
        x, y = [_f64(h) for h in o.split()]
        for got in (x, y):
            assert abs(Fraction(got) - exact) <= scale / 2 ** 51, (v, k, got)
        if k < 2:
            assert x == y == _round(exact), (v, k, x, y)


def test_float_float_split_of_fp64(harness):
    # the FP64 -> (hi, lo) split of the mixed Arnoldi basis: for 2^-74 <= |x| < 2^127 hi is x cut to 24 significant
    # bits and lo the rest rounded to FP32, |hi + lo - x| <= 2^-48 |x|; other x take the conversions
    # (hi = x rounded to FP32, lo = (x - hi) rounded to FP32)
    import numpy as np

    exe, _ = harness
    rng = random.Random(17)
    xs = [0.0, -0.0, 1.0, -1.0, 2.0 ** -74, 2.0 ** -75, 2.0 ** 127, 2.0 ** 127 * 1.5, 2.0 ** 128, 1e-300, 5e-324,
          float("inf"), float("-inf"), float("nan"), 1.0 + 2.0 ** -30, (1 << 53) - 1.0]
    for _ in range(30000):
        r = rng.random()
        if r < 0.8:
            x = rng.gauss(0, 1) * 2.0 ** rng.randint(-80, 130)
        else:
            x = struct.unpack("<d", struct.pack("<Q", rng.getrandbits(64)))[0]
        xs.append(x)
    lines = ["%016x" % struct.unpack("<Q", struct.pack("<d", x))[0] for x in xs]
    out = _run(exe, 3, lines)
    for x, o in zip(xs, out):
        hi, lo = [struct.unpack("<f", struct.pack("<I", int(h, 16)))[0] for h in o.split()]
        if x != x:
            assert hi != hi, o
            continue
        e = (struct.unpack("<Q", struct.pack("<d", x))[0] >> 52) & 0x7FF
        if 949 <= e <= 1150:
            err = abs(Fraction(hi) + Fraction(lo) - Fraction(x))
            assert err <= abs(Fraction(x)) / 2 ** 48, (x, hi, lo)
            assert abs(Fraction(hi)) <= abs(Fraction(x)) and (hi == 0.0) == (x == 0.0), (x, hi)
            assert abs(lo) <= abs(hi) * 2.0 ** -23, (x, hi, lo)
        else:
            with np.errstate(over="ignore", invalid="ignore"):
                want_hi = float(np.float32(x))
                want_lo = float(np.float32(x - want_hi)) if want_hi == want_hi and abs(want_hi) != float("inf") else None
            assert hi == want_hi or (hi != hi and want_hi != want_hi), (x, hi, want_hi)
            if want_lo is not None:
                assert lo == want_lo, (x, lo, want_lo)
