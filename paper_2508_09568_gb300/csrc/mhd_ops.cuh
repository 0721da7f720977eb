// Element operations of the scheme code (mhd_math.cuh), written as functions so that the
// arithmetic reads the same for float and double and states its roundings: fused
// multiply-adds are explicit, and region choices are selections rather than branches
// (comparisons give a mask, sel() picks).
//
// Helpers used by the scheme code for R = float, double:
//   fma_(a, b, c) = a * b + c rounded once      sel(m, a, b) = m ? a : b
//   mul_(a, b) = a * b, never fused
//   lt / le / gt / ge -> mask                   mand / mor / mnot on masks
//   rabs, rdiv (quotient), rsqrt_ (square root), fmax_ / fmin_ (larger / smaller value)
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#ifndef MHD_HD
#define MHD_HD __host__ __device__ __forceinline__
#endif

namespace mhd {

MHD_HD float fma_(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return fmaf(a, b, c);
#endif
}
MHD_HD double fma_(double a, double b, double c) {
#ifdef __CUDA_ARCH__
    return __fma_rn(a, b, c);
#else
    return fma(a, b, c);
#endif
}

// a * b rounded on its own: never fused into a neighbouring addition by the compiler, so
// that every kernel that evaluates the same expression rounds it the same way
MHD_HD float mul_(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
MHD_HD double mul_(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    return a * b;
#endif
}

template <typename R>
MHD_HD bool lt(R a, R b) { return a < b; }
template <typename R>
MHD_HD bool le(R a, R b) { return a <= b; }
template <typename R>
MHD_HD bool gt(R a, R b) { return a > b; }
template <typename R>
MHD_HD bool ge(R a, R b) { return a >= b; }
MHD_HD bool mand(bool a, bool b) { return a && b; }
MHD_HD bool mor(bool a, bool b) { return a || b; }
MHD_HD bool mnot(bool a) { return !a; }
template <typename R>
MHD_HD R sel(bool m, R a, R b) { return m ? a : b; }

// |x| (the sign of a zero result is +0; the scheme only compares magnitudes or divides
// them, so it never depends on that sign).  fabs lets the compiler fold |.| into the
// consuming instruction as an operand modifier instead of a compare and a select.
MHD_HD float rabs(float x) { return fabsf(x); }
MHD_HD double rabs(double x) { return fabs(x); }

MHD_HD float rsqrt_(float x) { return sqrtf(x); }
MHD_HD double rsqrt_(double x) { return sqrt(x); }

// Quotient.  Single precision on the device: the hardware approximate division
// (__fdividef: a reciprocal and a multiply, within 2 ulp for divisors below 2^126 in
// magnitude, which every divisor of the scheme is); double precision and host code: the
// IEEE operation.
MHD_HD float rdiv(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fdividef(a, b);
#else
    return a / b;
#endif
}
MHD_HD double rdiv(double a, double b) { return a / b; }

// x is finite (tested in its own precision: no conversion to double)
MHD_HD bool finite_(float x) { return isfinite(x); }
MHD_HD bool finite_(double x) { return isfinite(x); }

// Larger / smaller of two values (NaN operands are not propagated; the scheme's results
// are checked for finiteness where they are written).
MHD_HD float fmax_(float a, float b) { return fmaxf(a, b); }
MHD_HD float fmin_(float a, float b) { return fminf(a, b); }
MHD_HD double fmax_(double a, double b) { return fmax(a, b); }
MHD_HD double fmin_(double a, double b) { return fmin(a, b); }

}  // namespace mhd
