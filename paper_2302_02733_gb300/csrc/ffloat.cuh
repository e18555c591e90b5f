// FP32 building blocks of the mixed form's per-point work that use neither the FP64 pipe nor
// the conversion instructions.
//
// On GB300 the FP64 units issue 2 thread operations per clock per SM, and the FP64 geodesic
// keeps them busy; the FP32 transfer shares the SMs with it. So the transfer reads the FP64
// path through integer operations: a double becomes a pair of floats (value and remainder),
// and the few differences that need more than FP32's 24 bits (the grid fetch's cell fractions)
// are formed from such pairs with error-free FMA products (Dekker's two-product). Conversions
// between int and float (16 per clock per SM, an eighth of the FP32 rate) are replaced by the
// 1.5 * 2^23 offset, exact for magnitudes below 2^22.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace prt {

// double -> float rounded to nearest even with integer operations only. Magnitudes below the
// float normal range become signed zero; above it, infinity.
__device__ __forceinline__ float d2f_int(double d) {
    unsigned long long x = (unsigned long long)__double_as_longlong(d);
    unsigned hi = (unsigned)(x >> 32), lo = (unsigned)x;
    unsigned sign = hi & 0x80000000u;
    int fe = (int)((hi >> 20) & 0x7ffu) - 896;
    if (fe <= 0) return __uint_as_float(sign);
    if (fe >= 255) return __uint_as_float(sign | 0x7f800000u);
    unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
    unsigned rem = lo & 0x1fffffffu;
    unsigned f = sign | ((unsigned)fe << 23) | mant;
    f += (unsigned)(rem > 0x10000000u) | ((unsigned)(rem == 0x10000000u) & (mant & 1u));
    return __uint_as_float(f);
}

// float -> double, exact, with integer operations only (a conversion instruction would take the
// FP64 pipe). Zero and subnormal floats become signed zero; infinity and NaN keep their class.
__device__ __forceinline__ double f2d_int(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    if (e == 0u) return __longlong_as_double((long long)sign);
    const unsigned long long de = e == 0xffu ? 0x7ffull : (unsigned long long)(e + 896u);
    return __longlong_as_double((long long)(sign | (de << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}

// 2x and x/2 of a double, exactly as the FP64 sum x + x and product 0.5 x round them, with
// integer operations only (the FP64 pipe bounds the geodesic; the integer pipe is idle there).
// twice: a normal x below 2^1023 gets one more in its exponent field; a zero or subnormal x
// doubles its significand (carrying into the exponent field when it becomes normal); a larger x
// overflows to infinity; infinity and NaN pass through.
__device__ __forceinline__ double twice(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long e = b & 0x7ff0000000000000ull, sign = b & 0x8000000000000000ull;
    unsigned long long r;
    if (e == 0ull)
        r = sign | ((b & 0x000fffffffffffffull) << 1);
    else if (e >= 0x7fe0000000000000ull)
        r = e == 0x7ff0000000000000ull ? b : (sign | 0x7ff0000000000000ull);
    else
        r = b + (1ull << 52);
    return __longlong_as_double((long long)r);
}
// halve: a normal x with exponent field above 1 gets one less; otherwise the significand
// (with its implicit bit) is halved, rounded to nearest even; infinity and NaN pass through.
__device__ __forceinline__ double halve(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long e = b & 0x7ff0000000000000ull, sign = b & 0x8000000000000000ull;
    unsigned long long r;
    if (e >= (2ull << 52) && e != 0x7ff0000000000000ull) {
        r = b - (1ull << 52);
    } else if (e == 0x7ff0000000000000ull) {
        r = b;
    } else {
        const unsigned long long m = (b & 0x000fffffffffffffull) | (e ? (1ull << 52) : 0ull);
        unsigned long long q = m >> 1;
        q += (m & 1ull) & (q & 1ull);
        r = sign | q;
    }
    return __longlong_as_double((long long)r);
}

// The nearest integer of |x| < 2^22, and the float of an integer |i| < 2^22: adding
// 1.5 * 2^23 moves x into the binade whose unit in the last place is 1, where the mantissa
// bits hold round(x) in two's complement.
__device__ __forceinline__ int rint_small(float x) { return __float_as_int(x + 12582912.0f) - 0x4B400000; }
__device__ __forceinline__ float i2f_small(int i) { return __int_as_float(i + 0x4B400000) - 12582912.0f; }
// floor of |x| < 2^22
__device__ __forceinline__ int floor_small(float x) {
    int k = rint_small(x);
    return k - (i2f_small(k) > x ? 1 : 0);
}

// d = hi + lo: hi is d rounded to FP32 (as d2f_int), lo the remainder d - hi to about 2^-24
// of itself (the 29 bits below hi's last, as two exact 13- and 16-bit halves). For |d| in the
// FP32 normal range; lo becomes 0 for |d| below 2^-74 and hi for |d| outside the range.
__device__ __forceinline__ void split_ff(double d, float &hi, float &lo) {
    unsigned long long x = (unsigned long long)__double_as_longlong(d);
    unsigned hw = (unsigned)(x >> 32), lw = (unsigned)x;
    unsigned sign = hw & 0x80000000u;
    int e = (int)((hw >> 20) & 0x7ffu);
    int fe = e - 896;
    if (fe <= 0 || fe >= 255) {
        hi = d2f_int(d);
        lo = 0.0f;
        return;
    }
    unsigned mant = ((hw & 0xfffffu) << 3) | (lw >> 29);
    unsigned rem = lw & 0x1fffffffu;
    unsigned up = (unsigned)(rem > 0x10000000u) | ((unsigned)(rem == 0x10000000u) & (mant & 1u));
    hi = __uint_as_float((sign | ((unsigned)fe << 23) | mant) + up);
    // d - hi = sign * (rem - up 2^29) * 2^(e - 1075)
    int r = (int)rem - (int)(up << 29);
    unsigned ar = (unsigned)(r < 0 ? -r : r);
    float m = fmaf(i2f_small((int)(ar >> 16)), 65536.0f, i2f_small((int)(ar & 0xffffu)));
    int se = e - 1075 + 127;
    float sc = se > 0 ? __int_as_float(se << 23) : 0.0f;
    lo = ((r < 0) != (sign != 0u)) ? -(m * sc) : m * sc;
}

}  // namespace prt
