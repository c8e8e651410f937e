// df.cuh -- double-float arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.
// On this GPU an FP32 FMA issues at 64 times the FP64 rate, so a handful of
// FP32 operations per double-float operation is several times cheaper than
// one FP64 operation.  Built from the error-free transformations of
// floating-point sums and products: Knuth's TwoSum, the Dekker-style
// Fast2Sum for ordered operands, and the FMA form of TwoProduct
// (the product's rounding error is fma(a, b, -fl(a b))).  Host and device
// share the code, so the host tests check it against FP64 on the CPU.
#pragma once

#include <math.h>

namespace scvt {

#if defined(__CUDACC__)
#define SCVT_HD __host__ __device__ __forceinline__
#else
#define SCVT_HD inline
#endif

struct df {
    float hi, lo;
};

SCVT_HD float df_fma_f(float a, float b, float c) { return fmaf(a, b, c); }

// s + e == a + b exactly (any a, b)
SCVT_HD df two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return df{s, e};
}

// s + e == a + b exactly, |a| >= |b| (or a == 0)
SCVT_HD df fast_two_sum(float a, float b) {
    const float s = a + b;
    return df{s, b - (s - a)};
}

// p + e == a * b exactly (no underflow)
SCVT_HD df two_prod(float a, float b) {
    const float p = a * b;
    return df{p, df_fma_f(a, b, -p)};
}

SCVT_HD df df_from(double x) {
    const float h = (float)x;
    return df{h, (float)(x - (double)h)};
}

SCVT_HD double df_to(df x) { return (double)x.hi + (double)x.lo; }

SCVT_HD df df_neg(df x) { return df{-x.hi, -x.lo}; }

// x + y with error <= ~2^-47 (|x| + |y|): exact sum of the high parts, the
// low parts added in FP32.  Its error is relative to the operands, not to the
// result, which is what every sum here needs (no result is a small difference
// of large double-float operands whose relative accuracy matters)
SCVT_HD df df_add(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    s.lo += x.lo + y.lo;
    return fast_two_sum(s.hi, s.lo);
}

SCVT_HD df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

// x + f for an FP32 f
SCVT_HD df df_add_f(df x, float f) {
    df s = two_sum(x.hi, f);
    s.lo += x.lo;
    return fast_two_sum(s.hi, s.lo);
}

// x * y, relative error <= ~2^-46
SCVT_HD df df_mul(df x, df y) {
    df p = two_prod(x.hi, y.hi);
    p.lo = df_fma_f(x.hi, y.lo, p.lo);
    p.lo = df_fma_f(x.lo, y.hi, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

// x * f for an FP32 f
SCVT_HD df df_mul_f(df x, float f) {
    df p = two_prod(x.hi, f);
    p.lo = df_fma_f(x.lo, f, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

// x * y + z
SCVT_HD df df_fma(df x, df y, df z) { return df_add(df_mul(x, y), z); }

// x / y: the FP32 quotient refined by one Newton step on the remainder
SCVT_HD df df_div(df x, df y) {
    const float q1 = x.hi / y.hi;
    const df r = df_sub(x, df_mul_f(y, q1));
    const float q2 = r.hi / y.hi;
    return fast_two_sum(q1, q2);
}

// ---- unnormalized operations for chains of intermediate values: the same
// as df_add / df_mul without the closing Fast2Sum, so lo may grow to a few
// ulps of hi (hi + lo is the value).  Their errors stay of the same order
// while no sum cancels; a pair that comes out of a cancelling sum is
// normalized (df_norm) before it is multiplied, since the product takes only
// FP32 precision of lo.
SCVT_HD df df_norm(df x) { return fast_two_sum(x.hi, x.lo); }
SCVT_HD df dfl_add(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    s.lo += x.lo + y.lo;
    return s;
}
SCVT_HD df dfl_add_f(df x, float f) {
    df s = two_sum(x.hi, f);
    s.lo += x.lo;
    return s;
}
SCVT_HD df dfl_mul(df x, df y) {
    df p = two_prod(x.hi, y.hi);
    p.lo = df_fma_f(x.hi, y.lo, p.lo);
    p.lo = df_fma_f(x.lo, y.hi, p.lo);
    return p;
}
SCVT_HD df dfl_mul_f(df x, float f) {
    df p = two_prod(x.hi, f);
    p.lo = df_fma_f(x.lo, f, p.lo);
    return p;
}
SCVT_HD df dfl_fma(df x, df y, df z) { return dfl_add(dfl_mul(x, y), z); }

struct df3 {
    df x, y, z;
};

SCVT_HD df3 df3_from(double x, double y, double z) { return df3{df_from(x), df_from(y), df_from(z)}; }
// dot and cross products from unnormalized steps, the results normalized
SCVT_HD df df3_dot_n(df3 a, df3 b) {
    return df_norm(dfl_add(dfl_add(dfl_mul(a.x, b.x), dfl_mul(a.y, b.y)), dfl_mul(a.z, b.z)));
}
SCVT_HD df3 df3_cross_n(df3 a, df3 b) {
    return df3{df_norm(dfl_add(dfl_mul(a.y, b.z), df_neg(dfl_mul(a.z, b.y)))),
               df_norm(dfl_add(dfl_mul(a.z, b.x), df_neg(dfl_mul(a.x, b.z)))),
               df_norm(dfl_add(dfl_mul(a.x, b.y), df_neg(dfl_mul(a.y, b.x))))};
}
SCVT_HD df df3_dot(df3 a, df3 b) { return df_add(df_add(df_mul(a.x, b.x), df_mul(a.y, b.y)), df_mul(a.z, b.z)); }
SCVT_HD df3 df3_cross(df3 a, df3 b) {
    return df3{df_sub(df_mul(a.y, b.z), df_mul(a.z, b.y)), df_sub(df_mul(a.z, b.x), df_mul(a.x, b.z)),
               df_sub(df_mul(a.x, b.y), df_mul(a.y, b.x))};
}

#undef SCVT_HD

}  // namespace scvt
