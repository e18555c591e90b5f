"""The integer-pipe arithmetic of csrc/ffloat.cuh, compiled for the CPU and checked against the
host's IEEE arithmetic on random bit patterns and on the boundary cases of each function:
- twice(x) has the bits of x + x, and halve(x) those of 0.5 x, for every non-NaN double
  (subnormals, the largest normals, zeros and infinities included);
- d2f_int(d) is d rounded to the nearest FP32 value (ties to even), signed zero below the FP32
  normal range and infinity above it;
- f2d_int(f) is f widened exactly, signed zero for zero and subnormal f;
- rint_small, i2f_small and floor_small equal nearbyint, the int-to-float conversion and floor
  below 2^22;
- split_ff(d) gives hi = d2f_int(d) and lo within 2^-24 of the remainder d - hi.
The device versions are the same source. The GPU path leans on these identities where it
replaces FP64 instructions and conversions with integer operations. No GPU is used."""
import os
import shutil
import subprocess
import tempfile

import pytest

import __graft_entry__  # noqa: F401  (puts the repo root on sys.path)

SRC = r"""
// host build of the device header: an empty runtime header stands in, and the bit casts are
// shimmed
#include <cstdint>
#include <cstring>
#include <cmath>
#include <cstdio>
#include <cfloat>
#define __device__
#define __forceinline__ inline
static inline long long __double_as_longlong(double d) { long long x; std::memcpy(&x, &d, 8); return x; }
static inline double __longlong_as_double(long long x) { double d; std::memcpy(&d, &x, 8); return d; }
static inline unsigned __float_as_uint(float f) { unsigned u; std::memcpy(&u, &f, 4); return u; }
static inline float __uint_as_float(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }
static inline int __float_as_int(float f) { int i; std::memcpy(&i, &f, 4); return i; }
static inline float __int_as_float(int i) { float f; std::memcpy(&f, &i, 4); return f; }
#include "ffloat.cuh"
using namespace prt;

static uint64_t s = 0x9e3779b97f4a7c15ull;
static uint64_t next() {  // splitmix64
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
static uint64_t bits(double d) { uint64_t x; std::memcpy(&x, &d, 8); return x; }
static uint32_t fbits(float f) { uint32_t x; std::memcpy(&x, &f, 4); return x; }
static double dof(uint64_t x) { double d; std::memcpy(&d, &x, 8); return d; }
static float fof(uint32_t x) { float f; std::memcpy(&f, &x, 4); return f; }
static long bad = 0;
static void fail(const char *what, uint64_t x) {
    if (bad++ < 10) std::printf("FAIL %s %016llx\n", what, (unsigned long long)x);
}

static void check_double(uint64_t b) {
    const double x = dof(b);
    if (std::isnan(x)) {
        if (!std::isnan(twice(x)) || !std::isnan(halve(x))) fail("nan class", b);
        return;
    }
    volatile double two = 2.0, half = 0.5;
    if (bits(twice(x)) != bits(x * two)) fail("twice", b);
    if (bits(halve(x)) != bits(x * half)) fail("halve", b);
    const float f = d2f_int(x);
    const double ax = std::fabs(x);
    if (ax < (double)FLT_MIN) {
        if (fbits(f) != (std::signbit(x) ? 0x80000000u : 0u)) fail("d2f_int small", b);
    } else if (fbits(f) != fbits((float)x)) {
        fail("d2f_int", b);
    }
    if (std::isfinite(x) && ax >= (double)FLT_MIN && ax <= (double)FLT_MAX) {
        float hi, lo;
        split_ff(x, hi, lo);
        if (fbits(hi) != fbits(f)) fail("split_ff hi", b);
        if (std::isfinite(hi)) {
            const double rem = x - (double)hi;  // exact: the bits of x below hi's last
            const double tol = std::ldexp(std::fabs(rem), -24) + (ax < 0x1p-74 ? std::fabs(rem) : 0.0) + 0x1p-149;
            if (!(std::fabs((double)lo - rem) <= tol)) fail("split_ff lo", b);
        }
    }
}

static void check_float(uint32_t u) {
    const float f = fof(u);
    const double d = f2d_int(f);
    if (std::isnan(f)) {
        if (!std::isnan(d)) fail("f2d_int nan", u);
    } else if (std::fabs(f) < FLT_MIN) {
        if (bits(d) != (std::signbit(f) ? 0x8000000000000000ull : 0ull)) fail("f2d_int small", u);
    } else if (bits(d) != bits((double)f)) {
        fail("f2d_int", u);
    }
    if (std::fabs(f) < 4194304.0f) {  // 2^22
        if (rint_small(f) != (int)std::nearbyint(f)) fail("rint_small", u);
        if (floor_small(f) != (int)std::floor(f)) fail("floor_small", u);
    }
}

int main() {
    long n = 0;
    const uint64_t exps[] = {0x000, 0x001, 0x002, 0x380, 0x381, 0x382, 0x3ff, 0x47e, 0x47f, 0x7fd, 0x7fe, 0x7ff};
    const uint64_t mants[] = {0, 1, 2, 3, 0x0000000010000000ull, 0x0000000010000001ull, 0x000000001fffffffull,
                              0x0000000020000000ull, 0x0000000030000000ull, 0x000fffffe0000000ull,
                              0x000ffffff0000000ull, 0x000fffffffffffffull, 0x0008000000000000ull};
    for (uint64_t sg = 0; sg < 2; sg++)
        for (uint64_t e : exps)
            for (uint64_t m : mants) {
                check_double((sg << 63) | (e << 52) | m);
                n++;
            }
    for (long i = 0; i < (1l << 23); i++, n++) {
        uint64_t b = next();
        check_double(b);
        // exponents near the FP32 range and the subnormals, where the functions branch
        const uint64_t e = 0x36a + (next() % 0x120);
        check_double((b & 0x800fffffffffffffull) | (e << 52));
        check_double(b & 0x800fffffffffffffull);
    }
    for (uint64_t u = 0; u < (1ull << 32); u += 61) check_float((uint32_t)u);
    const uint32_t fspecial[] = {0u, 0x80000000u, 1u, 0x007fffffu, 0x00800000u, 0x7f7fffffu, 0x7f800000u,
                                 0xff800000u, 0x7fc00000u, 0x4a7fffffu, 0xca7fffffu, 0x3f000000u, 0xbf000000u,
                                 0x3fc00000u, 0x40200000u};
    for (uint32_t u : fspecial) check_float(u);
    for (int i = -4194303; i <= 4194303; i++)
        if (fbits(i2f_small(i)) != fbits((float)i)) fail("i2f_small", (uint64_t)(uint32_t)i);
    std::printf("doubles %ld failures %ld\n", n, bad);
    return bad != 0;
}
"""


def test_integer_pipe_arithmetic_matches_ieee():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    csrc = os.path.join(__graft_entry__.ROOT, "paper_2302_02733_gb300", "csrc")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "ffloat.cpp"), os.path.join(d, "ffloat")
        with open(src, "w") as f:
            f.write(SRC)
        with open(os.path.join(d, "cuda_runtime.h"), "w") as f:
            f.write("#pragma once\n")
        r = subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I", d, "-I", csrc, "-o", exe, src],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stdout + r.stderr
        assert "failures 0" in r.stdout
