// Device arithmetic helpers shared by the libmrcm kernels: FP64 <-> FP32
// conversions and an FP64 reciprocal that avoid the FP64 unit's slow paths.
#pragma once
#include <cuda_runtime.h>

namespace mrcm {

// FP64 <-> FP32 conversions on the integer pipe.  On this GPU a conversion
// instruction occupies the FP64 unit as long as an FMA does, and the local
// solve is bound by that unit, so the refinement loop converts with bit
// operations instead: FP64 -> FP32 truncates the significand (round toward
// zero; the FP32 value only feeds the low-precision correction solve),
// flushes magnitudes below the FP32 normal range to zero and saturates to
// infinity above it; FP32 -> FP64 is exact for normal numbers (FP32
// subnormals, which the correction never needs, become zero).
__device__ __forceinline__ float f64_to_f32_rz(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FF) - 1023 + 127;
    unsigned int f;
    if (e <= 0) f = sign;
    else if (e >= 255) f = sign | 0x7F800000u;
    else f = sign | ((unsigned int)e << 23) | (unsigned int)((b >> 29) & 0x7FFFFFu);
    return __uint_as_float(f);
}
__device__ __forceinline__ double f32_to_f64(float x) {
    const unsigned int f = __float_as_uint(x);
    const unsigned long long sign = (unsigned long long)(f & 0x80000000u) << 32;
    const int e = (int)((f >> 23) & 0xFF);
    unsigned long long b;
    if (e == 0) b = sign;
    else if (e == 255) b = sign | 0x7FF0000000000000ull | ((unsigned long long)(f & 0x7FFFFFu) << 29);
    else b = sign | ((unsigned long long)(e - 127 + 1023) << 52) | ((unsigned long long)(f & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)b);
}

// 1 / d by Newton-Raphson iteration y <- y + y (1 - d y) from an FP32 seed
// (FP32 reciprocal of d truncated to FP32, both conversions done with bit
// operations): each step squares the relative error, so two steps take the
// seed's ~2^-22 to the FP64 rounding level.  On this GPU an FP64 division is
// a ~470-cycle dependent chain on the FP64 unit, this one four FMAs.  Values
// whose reciprocal leaves the FP32 range fall back to the division.
__device__ __forceinline__ double rcp64(double d) {
    const unsigned long long bd = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((bd >> 52) & 0x7FF) - 1023;
    if (e < -125 || e > 125) return 1.0 / d;
    const float df = __uint_as_float((unsigned int)(bd >> 32) & 0x80000000u |
                                     (unsigned int)(e + 127) << 23 | (unsigned int)((bd >> 29) & 0x7FFFFFu));
    float yf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(df));
    const unsigned int fy = __float_as_uint(yf);
    const int ey = (int)((fy >> 23) & 0xFF);
    double y = __longlong_as_double((long long)((unsigned long long)(fy & 0x80000000u) << 32 |
                                                (unsigned long long)(ey - 127 + 1023) << 52 |
                                                (unsigned long long)(fy & 0x7FFFFFu) << 29));
    double r = fma(-d, y, 1.0);
    y = fma(y, r, y);
    r = fma(-d, y, 1.0);
    return fma(y, r, y);
}

// 1 / d from the same FP32 seed by one third-order step, y (1 + e + e^2) with
// e = 1 - d y: the seed's ~2^-22 error cubed lies below the FP64 rounding, at
// three dependent FMAs instead of four (for pivot chains).
__device__ __forceinline__ double rcp64c(double d) {
    const unsigned long long bd = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((bd >> 52) & 0x7FF) - 1023;
    if (e < -125 || e > 125) return 1.0 / d;
    const float df = __uint_as_float((unsigned int)(bd >> 32) & 0x80000000u |
                                     (unsigned int)(e + 127) << 23 | (unsigned int)((bd >> 29) & 0x7FFFFFu));
    float yf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(df));
    const unsigned int fy = __float_as_uint(yf);
    const int ey = (int)((fy >> 23) & 0xFF);
    const double y = __longlong_as_double((long long)((unsigned long long)(fy & 0x80000000u) << 32 |
                                                      (unsigned long long)(ey - 127 + 1023) << 52 |
                                                      (unsigned long long)(fy & 0x7FFFFFu) << 29));
    const double r = fma(-d, y, 1.0);
    return fma(y, fma(r, r, r), y);
}

}  // namespace mrcm
