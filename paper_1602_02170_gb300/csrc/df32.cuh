// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi)/2, giving about 46 significant bits on
// the FP32 pipes.  Built from the classic error-free transformations:
// Knuth's two-sum (the exact rounding error of a + b), the fast two-sum of
// Dekker for |a| >= |b|, and the exact product error of a * b obtained with a
// fused multiply-add.  The reciprocal square root takes the FP32 estimate and
// one Newton step y <- y + y (1 - x y^2) / 2, with the residual 1 - x y^2
// formed from exact products, which doubles the number of correct bits.
//
// GB300 runs FP64 at a small fraction of its FP32 rate; the pair kernel in
// double-float reaches FP64-class accuracy for the refinement residuals of
// the mixed-precision solver at a fraction of the FP64 kernel's time.
#pragma once

#include <cuda_runtime.h>

namespace mb {

struct dfl {
    float hi, lo;

    __host__ __device__ constexpr dfl() : hi(0.f), lo(0.f) {}
    __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    // exact split of a double into hi + lo (constant-folded for literals)
    __host__ __device__ constexpr dfl(double d)
        : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ constexpr dfl(int i) : dfl((double)i) {}
};

__device__ __forceinline__ dfl two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return dfl(s, e);
}

__device__ __forceinline__ dfl fast_two_sum(float a, float b)
{
    const float s = a + b;
    return dfl(s, b - (s - a));
}

// Addition in the "sloppy" form of Bailey's QD library (an exact two-sum of
// the high parts, the low parts added in FP32), here without the closing
// renormalisation: 8 FP32 operations instead of 20 for the form that also
// two-sums the low parts and renormalises twice.  The result hi + lo is not
// normalised (lo may exceed half an ulp of hi); every operation here accepts
// such operands, and subtraction, accumulation (+=) and the reciprocal square
// root renormalise.  The absolute error is within a few 2^-48 (|a| + |b|), so
// relative accuracy is lost only where a and b nearly cancel, and then only
// relative to the operands, which is what the pair sums need (about 1e-13 of
// each term).
__device__ __forceinline__ dfl operator+(dfl a, dfl b)
{
    const dfl s = two_sum(a.hi, b.hi);
    return dfl(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
// Subtraction renormalises: it forms the separations of nearby positions,
// where hi nearly cancels and the unnormalised lo would be large relative to
// the difference.
__device__ __forceinline__ dfl operator-(dfl a, dfl b)
{
    const dfl s = two_sum(a.hi, -b.hi);
    return fast_two_sum(s.hi, s.lo + (a.lo - b.lo));
}

// Product without the final renormalisation: lo may reach a few ulp of hi
// instead of half an ulp.  Every consumer (addition, product, conversion to
// double) takes such operands without loss beyond ~2^-46 relative.
__device__ __forceinline__ dfl operator*(dfl a, dfl b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return dfl(p, e);
}

// Accumulation renormalises (fast two-sum after the sloppy addition): a
// running sum over thousands of terms would otherwise let lo grow and lose
// bits in its FP32 additions.
__device__ __forceinline__ dfl &operator+=(dfl &a, dfl b)
{
    const dfl s = two_sum(a.hi, b.hi);
    a = fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
    return a;
}

// Products and sums with an FP32 operand c (a constant exact in FP32, or a
// value known to have no low part): the terms of c's absent low part are
// dropped.  a * c in 3 operations; a * 2^k exactly in 2; a + c in 7 (the
// sloppy form above with b.lo = 0).
__device__ __forceinline__ dfl mulf(dfl a, float c)
{
    const float p = a.hi * c;
    float e = fmaf(a.hi, c, -p);
    e = fmaf(a.lo, c, e);
    return dfl(p, e);
}

__device__ __forceinline__ dfl mul_pow2(dfl a, float c) { return dfl(a.hi * c, a.lo * c); }

__device__ __forceinline__ dfl addf(dfl a, float c)
{
    const dfl s = two_sum(a.hi, c);
    return dfl(s.hi, s.lo + a.lo);
}

// y^2 of an FP32 value as an exact double-float
__device__ __forceinline__ dfl sqf(float y)
{
    const float p = y * y;
    return dfl(p, fmaf(y, y, -p));
}

__device__ __forceinline__ bool operator<(dfl a, dfl b)
{
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

__device__ __forceinline__ dfl mb_max(dfl a, dfl b) { return a < b ? b : a; }

__device__ __forceinline__ dfl mb_rsqrt(dfl x)
{
    x = fast_two_sum(x.hi, x.lo);  // the FP32 estimate needs the normalised hi
    const float y0 = rsqrtf(x.hi);
    // r = 1 - x y0^2 (about 2^-22) to FP32 accuracy: y0^2 = s + t exactly,
    // x_hi s = p + e exactly, and 1 - p is exact (p is within 2^-21 of 1)
    const float s = y0 * y0, t = fmaf(y0, y0, -s);
    const float p = x.hi * s, e = fmaf(x.hi, s, -p);
    const float r = ((1.f - p) - e) - fmaf(x.hi, t, x.lo * s);
    // y = y0 + y0 r / 2
    return fast_two_sum(y0, (0.5f * y0) * r);
}

// Accumulation without renormalisation (the sloppy addition): for running
// sums that are renormalised, or converted to double, within a few dozen
// terms, so that lo stays within a few dozen ulp of hi.
__device__ __forceinline__ void acc_add(dfl &a, dfl b) { a = a + b; }
__device__ __forceinline__ void acc_add(float &a, float b) { a += b; }
__device__ __forceinline__ void acc_add(double &a, double b) { a += b; }
__device__ __forceinline__ void renorm(dfl &a) { a = fast_two_sum(a.hi, a.lo); }

__device__ __forceinline__ double to_double(dfl a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ float hi_part(dfl a) { return a.hi; }

}  // namespace mb
