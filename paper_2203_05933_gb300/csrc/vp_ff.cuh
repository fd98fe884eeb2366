// Float-float ("double-single") arithmetic for the FP32 pipes of sm_103a.
//
// A value is the unevaluated sum hi + lo of two IEEE floats. Sums use the
// TwoSum error-free transformation (Knuth), products the FMA-based TwoProd
// (exact residual of one float product); both keep about 48 significant bits.
// Results are left unnormalised (|lo| small next to |hi| but not necessarily
// below half an ulp of hi); ff_norm renormalises. All float operations are the
// explicit round-to-nearest intrinsics so the compiler cannot contract or
// reassociate them.
#pragma once

#include <cuda_runtime.h>

namespace vp {
namespace ff {

struct F {
    float h, l;
};

struct C {  // complex float-float
    F re, im;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ F from_double(double x)
{
    const float h = __double2float_rn(x);
    return F{h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double to_double(F a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ F norm(F a)
{
    const float s = __fadd_rn(a.h, a.l);
    return F{s, __fsub_rn(a.l, __fsub_rn(s, a.h))};
}

__device__ __forceinline__ F add(F a, F b)
{
    float s, e;
    two_sum(a.h, b.h, s, e);
    return F{s, __fadd_rn(e, __fadd_rn(a.l, b.l))};
}

__device__ __forceinline__ F neg(F a) { return F{-a.h, -a.l}; }

__device__ __forceinline__ F mul(F a, F b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return F{p, e};
}

// a * b + c
__device__ __forceinline__ F fma(F a, F b, F c) { return add(mul(a, b), c); }

__device__ __forceinline__ C cmul(C a, C b)
{
    return C{add(mul(a.re, b.re), neg(mul(a.im, b.im))), add(mul(a.re, b.im), mul(a.im, b.re))};
}

__device__ __forceinline__ C cadd(C a, C b) { return C{add(a.re, b.re), add(a.im, b.im)}; }

__device__ __forceinline__ C cnorm(C a) { return C{norm(a.re), norm(a.im)}; }

__device__ __forceinline__ C from_float4(float4 v) { return C{F{v.x, v.y}, F{v.z, v.w}}; }

__device__ __forceinline__ float4 to_float4(C a) { return make_float4(a.re.h, a.re.l, a.im.h, a.im.l); }

__device__ __forceinline__ C from_double2(double2 z) { return C{from_double(z.x), from_double(z.y)}; }

__device__ __forceinline__ double2 to_double2(C a) { return make_double2(to_double(a.re), to_double(a.im)); }

}  // namespace ff
}  // namespace vp
