// fp_bits.cuh -- conversions and power-of-two scalings done on the integer
// pipe.  B300 issues FP64 instructions (adds, multiplies, compares and the
// FP32 <-> FP64 conversions) at ~2 per clock per SM, 1/64 of its FP32 rate, so
// an elementwise kernel over 64M doubles pays ~0.1 ms per FP64 instruction per
// element: more than the HBM time of moving those doubles once.  The routines
// below are exact re-encodings of IEEE-754 bit patterns (no rounding beyond
// what the formats define) and hand the rare special operands (subnormals,
// infinities, NaN, results leaving the normal range) to the FP64 instruction.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.h"

namespace ccb {

// Rare-path fallbacks live in non-inlined functions: a call is a real branch,
// whereas an inlined FP64 multiply or conversion on a rarely taken side of a
// select is often executed speculatively for every element (if-conversion),
// which would put it back on the FP64 pipe.
static __device__ __noinline__ float d2f_slow(double x) { return __double2float_rn(x); }
static __device__ __noinline__ double dmul_slow(double x, double a) { return x * a; }

// double -> float, round to nearest even.  Normal results are formed from the
// bit pattern: the 29 dropped mantissa bits decide the rounding (ties to the
// even neighbour; a carry out of the mantissa bumps the exponent, which is the
// correctly rounded result, infinity included at the top of the range).
__device__ __forceinline__ float f64_to_f32_rn(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int hi = (unsigned int)(b >> 32), lo = (unsigned int)b;
    const unsigned int sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu);
    if (e == 0) return __uint_as_float(sign);             // zero, or a double subnormal (below every float)
    const int ef = e - 1023 + 127;
    if (ef <= 0 || ef >= 255) return d2f_slow(x);
    const unsigned int m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned int rem = lo & 0x1fffffffu;
    unsigned int f = sign | ((unsigned int)ef << 23) | m;
    if (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) f += 1u;
    return __uint_as_float(f);
}

// 2^k * (+-f) as a double, exact, integer operations only (alpha = +-2^k,
// |k| < 512, so every float -- subnormals included -- lands in the normal
// double range): a normal float's exponent is rebiased (127 -> 1023) and
// shifted by k and its 23 mantissa bits move to the top of the double's 52; a
// subnormal is normalised at its leading one; zeros keep their (flipped) sign;
// infinities and NaNs keep their payload.
__device__ __forceinline__ double f32_to_f64_pow2(float f, int kexp, uint32_t sflip) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    const uint32_t sign = (u & 0x80000000u) ^ sflip;
    uint32_t hi, lo;
    if (e - 1u < 254u) {
        hi = sign | ((uint32_t)((int)e + 896 + kexp) << 20) | (m >> 3);
        lo = m << 29;
    } else if (e == 255u) {
        hi = sign | 0x7ff00000u | (m >> 3);
        lo = m << 29;
    } else if (m == 0u) {
        hi = sign;
        lo = 0u;
    } else {
        const int p = 31 - __clz((int)m);                       // leading one of m: value = 2^(p-149) * 1.x
        const unsigned long long mm = ((unsigned long long)m << (52 - p)) & 0xfffffffffffffull;
        hi = sign | ((uint32_t)(p + 874 + kexp) << 20) | (uint32_t)(mm >> 32);
        lo = (uint32_t)mm;
    }
    return __hiloint2double((int)hi, (int)lo);
}

// alpha * (double)f: the integer path for alpha = +-2^k; a general alpha
// multiplies (callers that care choose between the two outside their loops)
__device__ __forceinline__ double f32_to_f64_scaled(float f, const Scale &s) {
    if (s.general) return dmul_slow((double)f, s.value);
    return f32_to_f64_pow2(f, s.kexp, s.sflip);
}

// alpha * x, exact for alpha = +-2^k when x and the result are normal
// (exponent field shift), and for +-1 or a zero (sign bit); subnormals,
// inf/NaN and range exits multiply.
__device__ __forceinline__ double scale_f64(double x, const Scale &s) {
    if (s.general) return dmul_slow(x, s.value);
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu);
    const int ee = e + s.kexp;
    if (e >= 1 && e <= 2046 && ee >= 1 && ee <= 2046)
        return __hiloint2double((int)((hi + ((uint32_t)s.kexp << 20)) ^ s.sflip), (int)lo);
    if (s.kexp == 0 || ((hi & 0x7fffffffu) | lo) == 0u)    // +-1, or a zero: sign only
        return __hiloint2double((int)(hi ^ s.sflip), (int)lo);
    return dmul_slow(x, s.value);
}
__device__ __forceinline__ double2 scale_f64(double2 x, const Scale &s) {
    return make_double2(scale_f64(x.x, s), scale_f64(x.y, s));
}

// alpha * acc of an epilogue, whatever the accumulator type
__device__ __forceinline__ double epi_scale(float acc, const Scale &s) { return f32_to_f64_scaled(acc, s); }
__device__ __forceinline__ double epi_scale(double acc, const Scale &s) { return scale_f64(acc, s); }
__device__ __forceinline__ double2 epi_scale(double2 acc, const Scale &s) { return scale_f64(acc, s); }

}  // namespace ccb
