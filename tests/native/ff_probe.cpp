// Host build of the two-float helpers used by the projection kernel, exported for the
// tests (compiled by the test with g++; no GPU involved).
#include "ffmath.cuh"

extern "C" void ff_dot3_plus(const float* r, float t, const float* x, float* out) {
    const csgs::ff::F2 v = csgs::ff::dot3_plus(r[0], r[1], r[2], t, x[0], x[1], x[2]);
    out[0] = v.hi;
    out[1] = v.lo;
}

extern "C" void ff_persp(float f, float ahi, float alo, float bhi, float blo, float c, float* out) {
    const csgs::ff::F2 v = csgs::ff::persp(f, {ahi, alo}, {bhi, blo}, c);
    out[0] = v.hi;
    out[1] = v.lo;
}
