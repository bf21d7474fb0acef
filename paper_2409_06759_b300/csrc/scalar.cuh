// scalar.cuh -- element-type helpers shared by the FP64 kernels: each kernel
// is written once over T = double or double2 (an interleaved complex double).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "fp_bits.cuh"
#include "kernels.h"

namespace ccb {

// ------------------------------------------------------------------ scalars
// The kernels below are written once over the element type T: double, or
// double2 holding an interleaved complex double (re, im).
__device__ __forceinline__ double ld(const double *p) { return __ldg(p); }
__device__ __forceinline__ double2 ld(const double2 *p) { return __ldg(p); }
__device__ __forceinline__ double neg(double x) {           // sign bit only (no FP64 instruction)
    return __hiloint2double(__double2hiint(x) ^ (int)0x80000000, __double2loint(x));
}
__device__ __forceinline__ double2 neg(double2 x) { return make_double2(neg(x.x), neg(x.y)); }
__device__ __forceinline__ double cj(double x, int) { return x; }
__device__ __forceinline__ double2 cj(double2 x, int c) { return c ? make_double2(x.x, neg(x.y)) : x; }
__device__ __forceinline__ double mul(double a, double b) { return a * b; }
__device__ __forceinline__ double2 mul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// acc + s * x, s real
__device__ __forceinline__ double axpy(double s, double x, double acc) { return fma(s, x, acc); }
__device__ __forceinline__ double2 axpy(double s, double2 x, double2 acc) {
    return make_double2(fma(s, x.x, acc.x), fma(s, x.y, acc.y));
}
__device__ __forceinline__ double scal(double s, double x) { return s * x; }
__device__ __forceinline__ double2 scal(double s, double2 x) { return make_double2(s * x.x, s * x.y); }
template <typename T> __device__ __forceinline__ T zero();
template <> __device__ __forceinline__ double zero<double>() { return 0.0; }
template <> __device__ __forceinline__ double2 zero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float zero<float>() { return 0.0f; }
// element type T -> compute type CT (FP64 data multiplied in FP32: one rounding) and back
template <typename CT> __device__ __forceinline__ CT down(double x);
template <> __device__ __forceinline__ double down<double>(double x) { return x; }
template <> __device__ __forceinline__ float down<float>(double x) { return f64_to_f32_rn(x); }
template <typename CT> __device__ __forceinline__ CT down(double2 x) { return x; }
__device__ __forceinline__ double up(double x) { return x; }
__device__ __forceinline__ double up(float x) { return f32_to_f64_pow2(x, 0, 0u); }
__device__ __forceinline__ double2 up(double2 x) { return x; }
__device__ __forceinline__ float cfma(float a, float b, float acc) { return fmaf(a, b, acc); }
// B300's FP64 pipe issues ~2 operations per clock per SM: the elementwise
// kernels spend at most one FP64 operation per term.  A +-1 sign is an add or
// a subtract (the first term a free negation); alpha = +-1 and beta in {0, 1}
// cost nothing or one add.
__device__ __forceinline__ double add(double a, double b) { return a + b; }
__device__ __forceinline__ double2 add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double sub(double a, double b) { return a - b; }
__device__ __forceinline__ double2 sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
// acc (+|-) x, the first term taken as +-x
// (the sign is applied on the integer pipe, so a term is one add however the
// compiler resolves the selects)
template <typename T> __device__ __forceinline__ T signed_term(bool first, bool negative, T x, T acc) {
    const T sx = negative ? neg(x) : x;
    return first ? sx : add(acc, sx);
}
// alpha * acc (+ old when ACC, i.e. beta = 1): alpha = +-2^k on the integer
// pipe, so at most one FP64 add.  A general beta is applied beforehand by a
// separate scaling pass (the kernels are compiled for beta in {0, 1} only).
template <bool ACC, typename T> __device__ __forceinline__ T finish(const Scale &as, T acc, const T &old) {
    const T v = scale_f64(acc, as);
    return ACC ? add(v, old) : v;
}
// *p += v by a fire-and-forget reduction in L2 (no value returns to the SM)
__device__ __forceinline__ void red_add(double *p, double v) {
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void red_add(double2 *p, double2 v) {
    red_add(reinterpret_cast<double *>(p), v.x);
    red_add(reinterpret_cast<double *>(p) + 1, v.y);
}
// acc + a * b over complex (or real) numbers
__device__ __forceinline__ double cfma(double a, double b, double acc) { return fma(a, b, acc); }
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}

}  // namespace ccb
