// Two-float ("float-float") arithmetic for the projection of Gaussian means: error-free
// transformations (Dekker's product via FMA, Knuth's two-sum) and the compensated dot
// product Dot2 of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J. Sci.
// Comput. 26(6), 2005).  Every operation is explicitly rounded to nearest so that no
// contraction or reassociation can change the result.  Host and device share the
// definitions; the host versions let the tests check them against exact arithmetic.
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define CSGS_HD __host__ __device__ __forceinline__
#else
#define CSGS_HD inline
#endif

namespace csgs {
namespace ff {

CSGS_HD float add(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    volatile float r = a + b;
    return r;
#endif
}
CSGS_HD float sub(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    volatile float r = a - b;
    return r;
#endif
}
CSGS_HD float mul(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    volatile float r = a * b;
    return r;
#endif
}
CSGS_HD float fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return ::fmaf(a, b, c);
#endif
}
CSGS_HD float div(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fdiv_rn(a, b);
#else
    volatile float r = a / b;
    return r;
#endif
}

struct F2 {
    float hi, lo;
};

// p + e = a * b exactly
CSGS_HD F2 two_prod(float a, float b) {
    const float p = mul(a, b);
    return {p, fma(a, b, -p)};
}
// s + e = a + b exactly
CSGS_HD F2 two_sum(float a, float b) {
    const float s = add(a, b);
    const float bb = sub(s, a);
    return {s, add(sub(a, sub(s, bb)), sub(b, bb))};
}
// s + e = a + b exactly, given |a| >= |b| (or a = 0)
CSGS_HD F2 fast_two_sum(float a, float b) {
    const float s = add(a, b);
    return {s, sub(b, sub(s, a))};
}

// r0 x + r1 y + r2 z + t as a two-float value (Dot2 with the constant folded in)
CSGS_HD F2 dot3_plus(float r0, float r1, float r2, float t, float x, float y, float z) {
    F2 p = two_prod(r0, x);
    float h = p.hi, s = p.lo;
    F2 q = two_prod(r1, y);
    F2 u = two_sum(h, q.hi);
    h = u.hi;
    s = add(s, add(u.lo, q.lo));
    q = two_prod(r2, z);
    u = two_sum(h, q.hi);
    h = u.hi;
    s = add(s, add(u.lo, q.lo));
    u = two_sum(h, t);
    h = u.hi;
    s = add(s, u.lo);
    return two_sum(h, s);  // h may cancel to below |s|, so not the fast variant
}

// f * (a / b) + c for two-float a, b (b > 0), as a two-float value
CSGS_HD F2 persp(float f, F2 a, F2 b, float c) {
    const float q1 = div(a.hi, b.hi);
    float r = fma(-q1, b.hi, a.hi);  // exact remainder a.hi - q1 b.hi
    r = add(r, a.lo);
    r = fma(-q1, b.lo, r);
    const float q2 = div(r, b.hi);
    const F2 p = two_prod(f, q1);
    const float e = fma(f, q2, p.lo);
    const F2 s = two_sum(p.hi, c);
    const float lo = add(s.lo, e);
    // |s.hi| may be smaller than |lo| only when the sum cancels; use the general sum
    return two_sum(s.hi, lo);
}

}  // namespace ff
}  // namespace csgs
