// fr_ff.cuh -- float-float ("double-single") arithmetic for the FP64 mass channel of the low-Mach
// FP32 form. A value is the unevaluated sum hi + lo of two floats (|lo| <= ulp(hi)/2), about 48
// significant bits. Built from the error-free transformations of the floating-point literature:
// Knuth's TwoSum (exact sum of two floats), Dekker's FastTwoSum (the same when |a| >= |b|), and the
// exact product of two floats with one fused multiply-add (Ogita, Rump and Oishi, "Accurate sum and
// dot product", SIAM J. Sci. Comput. 26, 2005). GB300 issues FP32 about 70 times faster than FP64,
// so these few FP32 operations per step cost less than one FP64 operation.
#pragma once

struct ff {
    float hi, lo;
};

__host__ __device__ inline ff ff_from_double(double d)
{
    const float h = (float)d;
    return ff{h, (float)(d - (double)h)};
}

#ifdef __CUDACC__
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ ff ff_of(float a) { return ff{a, 0.0f}; }

// Knuth's TwoSum: s + e = a + b exactly.
__device__ __forceinline__ ff two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff{s, e};
}

// Dekker's FastTwoSum (|a| >= |b| or a = 0): s + e = a + b exactly.
__device__ __forceinline__ ff fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e = a b exactly (one fused multiply-add).
__device__ __forceinline__ ff two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return ff{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    ff s = two_sum(a.hi, b.hi);
    const float t = __fadd_rn(__fadd_rn(a.lo, b.lo), s.lo);
    return fast_two_sum(s.hi, t);
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

// a * f for a float f
__device__ __forceinline__ ff ff_mul_f(ff a, float f)
{
    ff p = two_prod(a.hi, f);
    return fast_two_sum(p.hi, __fmaf_rn(a.lo, f, p.lo));
}

__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    ff p = two_prod(a.hi, b.hi);
    const float t = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, t);
}

// acc + a * b
__device__ __forceinline__ ff ff_fma(ff a, ff b, ff acc) { return ff_add(acc, ff_mul(a, b)); }
__device__ __forceinline__ ff ff_fma_f(ff a, float f, ff acc) { return ff_add(acc, ff_mul_f(a, f)); }

// Compensated dot product sum_i a_i x_i of float-float coefficients and floats (Dot2 of Ogita, Rump
// and Oishi, with each coefficient's low part folded into the correction): s carries the TwoSum of
// the exact products' high parts, c their rounding errors, the TwoSum errors and lo(a_i) x_i; the
// value is two_sum(s, c), as accurate as a sum formed in twice the working precision. About two
// thirds of the operations of accumulating with ff_fma_f. Where the sum is rounded to one float at
// the end (face values), fast_two_sum(s, c) serves: its high part is the correctly rounded s + c
// whatever the magnitudes, and its low part can be inexact only when the sum has cancelled to below
// the rounding errors already in c.
__device__ __forceinline__ void dot2_first(ff a, float x, float &s, float &c)
{
    s = __fmul_rn(a.hi, x);
    c = __fmaf_rn(a.lo, x, __fmaf_rn(a.hi, x, -s));
}
__device__ __forceinline__ void dot2_next(ff a, float x, float &s, float &c)
{
    const float p = __fmul_rn(a.hi, x);
    const float e = __fmaf_rn(a.hi, x, -p);
    const ff t = two_sum(s, p);
    s = t.hi;
    c = __fmaf_rn(a.lo, x, __fadd_rn(c, __fadd_rn(e, t.lo)));
}
// One term with float-float factors on both sides: the cross products hi lo and lo hi go into the
// correction (lo lo, below 2^-48 of the product, is dropped, as ff_mul drops it). Start from s = hi,
// c = lo of an initial value (or zeros).
__device__ __forceinline__ void dot2ff_next(ff a, ff b, float &s, float &c)
{
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.hi, -p);
    const ff t = two_sum(s, p);
    s = t.hi;
    c = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, __fadd_rn(c, __fadd_rn(e, t.lo))));
}
#endif
