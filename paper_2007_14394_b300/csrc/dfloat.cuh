// Double-float arithmetic for the per-frame texel-weight table.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2: the
// "double-length" arithmetic of Dekker (1971) with Knuth's error-free two-sum and the
// fused multiply-add two-product, good to about 2^-44 relative. The cosine weights of
// Eq. 3 are computed in it so that a weight near the cosine cutoff keeps its relative
// accuracy: a float32 dot product of float32 directions carries an absolute error of
// about 1e-7, which is a large relative error on a ray that grazes a texel's horizon and
// then dominates that texel when it is the only lit ray it sees. No FP64 is used.
//
// The functions must not be compiled with reassociation (no fast-math): the error terms
// are exact differences that reassociation would fold to zero.
#pragma once

#include <cstdint>

namespace sdfddgi {

struct dfloat {
    float hi, lo;
};

__host__ __device__ constexpr dfloat df(float a) { return {a, 0.f}; }

// s + e == a + b exactly (Knuth).
__device__ __forceinline__ dfloat two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

// s + e == a + b exactly when |a| >= |b| or a == 0 (Dekker).
__device__ __forceinline__ dfloat quick_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}

// p + e == a * b exactly (the rounding error of a product is one fused multiply-add away).
__device__ __forceinline__ dfloat two_prod(float a, float b) {
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
    dfloat s = two_sum(a.hi, b.hi);
    const dfloat t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dfloat operator-(dfloat a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }

__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
    dfloat p = two_prod(a.hi, b.hi);
    p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
    return quick_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ dfloat operator*(dfloat a, float b) {
    dfloat p = two_prod(a.hi, b);
    p.lo = fmaf(a.lo, b, p.lo);
    return quick_two_sum(p.hi, p.lo);
}

// a / b: a float quotient, then one correction from the exact remainder a - q b.
__device__ __forceinline__ dfloat operator/(dfloat a, dfloat b) {
    const float q1 = a.hi / b.hi;
    const dfloat r = a - b * q1;
    const float q2 = r.hi / b.hi;
    return quick_two_sum(q1, q2);
}

// sqrt(m) of a nonnegative float m: the float root s, then one Newton correction from the
// exact residual m - s^2.
__device__ __forceinline__ dfloat df_sqrt(float m) {
    if (!(m > 0.f)) return df(0.f);
    const float s = sqrtf(m);
    const float e = fmaf(-s, s, m);
    return quick_two_sum(s, e / (2.f * s));
}

// A real constant as a double-float: the nearest float and the float nearest the remainder,
// evaluated by the compiler (constexpr) in double precision; nothing of it runs on the GPU.
__host__ __device__ constexpr dfloat df_const(double x) { return {(float)x, (float)(x - (double)(float)x)}; }

// cos and sin of 2 pi k / 2^32 for a 32-bit fixed-point turn k (the spherical-Fibonacci
// azimuth). The reduction is exact integer arithmetic: q = the nearest quarter turn, and
// the remainder r = k - q 2^30 (|r| <= 2^29) gives an angle a = 2 pi r / 2^32 in
// [-pi/4, pi/4]. sin a and cos a come from their Taylor series in Horner form (terms up to
// a^13 and a^14: truncation below 1e-12 on that interval), then the quarter turns rotate them.
__device__ __forceinline__ void df_sincos_turn(uint32_t k, dfloat* s_out, dfloat* c_out) {
    const uint32_t q = (k + (1u << 29)) >> 30;  // 0..4, taken mod 4 below
    const int32_t r = (int32_t)(k - (q << 30));
    // r as an exact double-float: high part a multiple of 256 (at most 22 bits), low part in [0, 255]
    const int32_t r_hi = (r >> 8) * 256;
    const dfloat rr = two_sum((float)r_hi, (float)(r - r_hi));
    // 2 pi / 2^32 as a double-float: the float nearest 2 pi and its remainder, scaled exactly
    const dfloat turn = {6.28318548202514648438f * 0x1p-32f, -1.7484555314695172e-07f * 0x1p-32f};
    const dfloat a = rr * turn;
    const dfloat a2 = a * a;
    // Taylor coefficients (-1)^j / (2j+1)! of sin a / a and (-1)^j / (2j)! of cos a
    constexpr dfloat s1 = df_const(-1.0 / 6.0), s2 = df_const(1.0 / 120.0), s3 = df_const(-1.0 / 5040.0),
                     s4 = df_const(1.0 / 362880.0), s5 = df_const(-1.0 / 39916800.0),
                     s6 = df_const(1.0 / 6227020800.0);
    constexpr dfloat c1 = df_const(-1.0 / 2.0), c2 = df_const(1.0 / 24.0), c3 = df_const(-1.0 / 720.0),
                     c4 = df_const(1.0 / 40320.0), c5 = df_const(-1.0 / 3628800.0),
                     c6 = df_const(1.0 / 479001600.0), c7 = df_const(-1.0 / 87178291200.0);
    dfloat sn = s5 + a2 * s6;
    sn = s4 + a2 * sn;
    sn = s3 + a2 * sn;
    sn = s2 + a2 * sn;
    sn = s1 + a2 * sn;
    sn = (df(1.f) + a2 * sn) * a;
    dfloat cs = c6 + a2 * c7;
    cs = c5 + a2 * cs;
    cs = c4 + a2 * cs;
    cs = c3 + a2 * cs;
    cs = c2 + a2 * cs;
    cs = c1 + a2 * cs;
    cs = df(1.f) + a2 * cs;
    switch (q & 3u) {
        case 0: *s_out = sn; *c_out = cs; break;
        case 1: *s_out = cs; *c_out = -sn; break;
        case 2: *s_out = -sn; *c_out = -cs; break;
        default: *s_out = -cs; *c_out = sn; break;
    }
}

// Spherical-Fibonacci direction i of R rotated by the float32 frame rotation rot (row
// major), in double-float: z = 1 - (2i+1)/R, radius sqrt((2i+1)(2R-2i-1))/R (an integer
// under the root, exact in float for R <= 2^11), azimuth 2 pi ((i * 2654435769) mod 2^32) / 2^32.
__device__ __forceinline__ void df_ray_direction(int i, int R, const float rot[9], dfloat d[3]) {
    const dfloat inv_r = df(1.f) / df((float)R);
    const dfloat z = df((float)(R - 2 * i - 1)) * inv_r;
    const dfloat rxy = df_sqrt((float)(2 * i + 1) * (float)(2 * R - 2 * i - 1)) * inv_r;
    dfloat s, c;
    df_sincos_turn((uint32_t)i * 2654435769u, &s, &c);
    const dfloat v[3] = {rxy * c, rxy * s, z};
    for (int r = 0; r < 3; ++r) d[r] = v[0] * rot[3 * r] + v[1] * rot[3 * r + 1] + v[2] * rot[3 * r + 2];
}

// Direction of interior texel (a, b) of an n x n octahedral map (pole +z), in double-float.
// The unnormalised octahedral point is an integer vector over n: x = 2a+1-n, y = 2b+1-n,
// z = n - |x| - |y|, folded for z < 0 to ((n - |y|) sign x, (n - |x|) sign y, z); the
// direction is that vector over its (integer) squared length's root.
__device__ __forceinline__ void df_texel_direction(int a, int b, int n, dfloat u[3]) {
    int x = 2 * a + 1 - n, y = 2 * b + 1 - n;
    const int z = n - abs(x) - abs(y);
    if (z < 0) {
        const int fx = (n - abs(y)) * (x >= 0 ? 1 : -1);
        const int fy = (n - abs(x)) * (y >= 0 ? 1 : -1);
        x = fx;
        y = fy;
    }
    const dfloat inv = df(1.f) / df_sqrt((float)(x * x + y * y + z * z));
    u[0] = inv * (float)x;
    u[1] = inv * (float)y;
    u[2] = inv * (float)z;
}

__device__ __forceinline__ dfloat df_dot(const dfloat a[3], const dfloat b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// c^p by binary powering, p >= 1.
__device__ __forceinline__ dfloat df_pow(dfloat c, int p) {
    dfloat r = df(1.f), b = c;
    while (p) {
        if (p & 1) r = r * b;
        b = b * b;
        p >>= 1;
    }
    return r;
}

}  // namespace sdfddgi
