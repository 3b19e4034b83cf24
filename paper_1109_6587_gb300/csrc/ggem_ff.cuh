// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2, about 48 significant bits.  GB300 issues
// FP64 at 1/64 of its FP32 rate, so FP64-accurate pair sums run faster in
// float pairs than in doubles.  Built on Knuth's two-sum and the exact product
// of a fused multiply-add (a*b - fl(a*b) = fma(a, b, -fl(a*b))); the addition
// and multiplication follow the published double-double algorithms of Dekker
// (1971) and Hida, Li and Bailey (2001), applied to float pairs.  Additions use
// the short ("sloppy") form: the error is about 2^-44 of the larger operand,
// which the pair sums tolerate (FP64 parity is checked at 1e-10).
#pragma once

struct ff {
    float hi, lo;
};

// FP64 -> pair (setup code only: it issues FP64 instructions)
__device__ __forceinline__ ff ff_from_double(double x) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ ff ff_of(float a) { return {a, 0.f}; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}
// p + e = a * b exactly
__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    ff s = two_sum(a.hi, b);
    s.lo += a.lo;
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    ff p = two_prod(a.hi, b.hi);
    p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
    ff p = two_prod(a.hi, b);
    p.lo = fmaf(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}
// a < b
__device__ __forceinline__ bool ff_lt(ff a, ff b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

// 1/sqrt(x), x > 0: the hardware estimate y (about 2^-23 relative) and one
// Newton step y + y (1 - x y^2)/2 with the residual 1 - x y^2 formed in pairs
__device__ __forceinline__ ff ff_rsqrt(ff x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x.hi));
    const ff t = ff_mul(x, two_prod(y, y));
    const ff e = ff_add_f(ff_neg(t), 1.0f);
    return fast_two_sum(y, 0.5f * y * (e.hi + e.lo));
}

// exp(x) for -20 <= x <= 0.  Reduction x = (16 m + j) ln2/16 + f, |f| <=
// ln2/32, exp(x) = 2^m 2^(j/16) exp(f); exp(f) = 1 + f + f^2/2 + f^3/6 in
// pairs plus the tail f^4 (1/24 + f/120 + f^2/720 + f^3/5040) in float (the
// tail is below 1e-8, its float rounding below 1e-15).  t2[j] = 2^(j/16),
// ln2_16 = ln 2 / 16 and sixth = 1/6 as pairs.
__device__ __forceinline__ ff ff_exp(ff x, const ff* t2, ff ln2_16, ff sixth) {
    const float kf = rintf(x.hi * 23.083120654223414f);   // 16 / ln 2
    const int k = (int)kf;
    const int m = k >> 4, j = k - 16 * m;
    ff kl = two_prod(kf, ln2_16.hi);
    kl.lo = fmaf(kf, ln2_16.lo, kl.lo);
    const ff f = ff_sub(x, kl);
    const ff f2 = ff_mul(f, f);
    const ff f3 = ff_mul(f2, f);
    ff h = ff_add(ff_add_f(f, 1.0f), ff_mul_f(f2, 0.5f));
    h = ff_add(h, ff_mul(f3, sixth));
    const float fh = f.hi, f4 = f2.hi * f2.hi;
    const float tail =
        f4 * fmaf(fh, fmaf(fh, fmaf(fh, 1.0f / 5040.0f, 1.0f / 720.0f), 1.0f / 120.0f),
                  1.0f / 24.0f);
    ff r = ff_mul(ff_add_f(h, tail), t2[j]);
    r.hi = ldexpf(r.hi, m);
    r.lo = ldexpf(r.lo, m);
    return r;
}
