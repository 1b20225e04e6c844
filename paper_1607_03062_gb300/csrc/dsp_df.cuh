// dsp_df.cuh -- double-float helpers and the density partial sums, shared by the
// kernels and the allocation-free density (not installed).
//
// A double-float value is an unevaluated pair hi + lo of floats (about 48
// significant bits).  Conversions between double and float are written with
// integer operations: on GB300 a cvt between FP64 and FP32 issues on the FP64
// pipe, at the FP64 rate.  Everything here is written from the definitions
// (TwoSum, IEEE-754 bit layouts) with non-contracting intrinsics, so every
// kernel that calls it gets the same bits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dsp_internal.h"

namespace dsp {

// s + e = a + b exactly (TwoSum, no condition on the magnitudes).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fadd_rn(s, -a);
    e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
}

// The double x as hi + lo floats: hi = x truncated to 24 significant bits (the
// same exponent as x), lo = the 29 fraction bits hi drops, rounded to a float
// (x - hi - lo is below 2^-48 |x|).  Values below 2^-126 in magnitude give
// hi = lo = 0 (an error below 2^-126); lo = 0 when |x| < 2^-74 (it is below
// 2^-97 then); |x| >= 2^128 gives an infinite hi, NaN a NaN.
__device__ __forceinline__ void split_f64(double x, float &hi, float &lo)
{
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned int top = static_cast<unsigned int>(b >> 32);
    const unsigned int low = static_cast<unsigned int>(b);
    const unsigned int e = (top >> 20) & 0x7FFu;  // biased exponent
    const unsigned int sign = top & 0x80000000u;
    const unsigned int m23 = ((top & 0xFFFFFu) << 3) | (low >> 29);
    lo = 0.0f;
    if (e < 897u) {
        hi = __uint_as_float(sign);
    } else if (e <= 1150u) {
        hi = __uint_as_float(sign | ((e - 896u) << 23) | m23);
        if (e >= 949u)  // scale 2^(e - 1075) is a normal float
            lo = __uint_as_float(sign ^ __float_as_uint(__fmul_rn(
                     __uint2float_rn(low & 0x1FFFFFFFu), __uint_as_float((e - 948u) << 23))));
    } else {
        const bool nan = e == 0x7FFu && ((top & 0xFFFFFu) | low) != 0u;
        hi = __uint_as_float(sign | 0x7F800000u | (nan ? 0x400000u : 0u));
    }
}

// The float f as a double, exactly (float subnormals, below 1.2e-38, become 0).
__device__ __forceinline__ double f32_to_f64(float f)
{
    const unsigned int u = __float_as_uint(f);
    const unsigned int e = (u >> 23) & 0xFFu;
    unsigned long long d = static_cast<unsigned long long>(u & 0x80000000u) << 32;
    const unsigned long long m = static_cast<unsigned long long>(u & 0x7FFFFFu) << 29;
    if (e == 0xFFu)
        d |= 0x7FF0000000000000ull | m;
    else if (e != 0u)
        d |= (static_cast<unsigned long long>(e + 896u) << 52) | m;
    return __longlong_as_double(static_cast<long long>(d));
}

// hi + lo rounded to a double (one FP64 add).
__device__ __forceinline__ double df_to_f64(float hi, float lo)
{
    return __dadd_rn(f32_to_f64(hi), f32_to_f64(lo));
}

// (h, l) <- (h, l) + (h2, l2) in double-float: TwoSum of the high parts, the low
// parts added to its error, then renormalised (relative error ~2^-46).
__device__ __forceinline__ void df_add(float &h, float &l, float h2, float l2)
{
    float s, e;
    two_sum(h, h2, s, e);
    e = __fadd_rn(e, __fadd_rn(l, l2));
    h = __fadd_rn(s, e);
    l = __fadd_rn(e, -__fadd_rn(h, -s));
}

// (ph, pl) = (ah + al)(bh + bl) to ~2^-46 relative: the high product split
// exactly by FMA, the cross terms added, then renormalised (Fast2Sum: |p| >= |e|).
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &ph, float &pl)
{
    const float p = __fmul_rn(ah, bh);
    const float e = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, __fmaf_rn(ah, bh, -p)));
    ph = __fadd_rn(p, e);
    pl = __fadd_rn(e, -__fadd_rn(ph, -p));
}

// The double c as a hi + lo pair of floats (rounded to nearest; compile time).
struct DFConst {
    float h, l;
};
__host__ __device__ constexpr DFConst df_const(double c)
{
    return DFConst{static_cast<float>(c),
                   static_cast<float>(c - static_cast<double>(static_cast<float>(c)))};
}

// Density partial sums, one per granule of kGranule consecutive points (point
// index / kGranule): red holds n_gran granules of kGranule double-float slots
// (slot k of a granule = its point k; zero for points past the grid's end).
// Each granule is summed by a fixed pairwise tree in double-float, then
// rounded to a double; granule indices come from gran_index(g).  Every kernel
// sums the same values in the same order, so the density does not depend on
// which kernel, tiling or batch produced them.
template <typename GranIndex>
__device__ __forceinline__ void granule_sums(float2 *red, int n_gran, double *partials,
                                             int64_t n_parts, GranIndex gran_index)
{
    __syncthreads();
    for (int s = kGranule / 2; s > 0; s >>= 1) {
        const int sh = __ffs(s) - 1;
        for (int i = threadIdx.x; i < n_gran * s; i += blockDim.x) {
            const int g = i >> sh, j = i & (s - 1);
            float2 &a = red[g * kGranule + j];
            const float2 b = red[g * kGranule + j + s];
            df_add(a.x, a.y, b.x, b.y);
        }
        __syncthreads();
    }
    if (static_cast<int>(threadIdx.x) < n_gran) {
        const int64_t gi = gran_index(static_cast<int>(threadIdx.x));
        if (gi < n_parts)
            partials[gi] = df_to_f64(red[threadIdx.x * kGranule].x, red[threadIdx.x * kGranule].y);
    }
}

}  // namespace dsp
