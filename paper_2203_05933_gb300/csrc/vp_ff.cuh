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

namespace vp {
namespace ff {

// ln 2 split for the exponent term of the table log: kLn2Hi has 19 fractional
// bits, so e * kLn2Hi + T_hi is exact in one float for |e| <= 15.
constexpr float kLn2Hi = 363409.0f / 524288.0f;
constexpr float kLn2Lo = (float)(0.693147180559945309417232121458176568 - 363409.0 / 524288.0);

// log(x) for x = xh + xl with 2^-15 <= xh < 2^16 (the caller checks), as
// (S, lo) with S + lo accurate to about 1.3e-12 absolute: x = 2^e m (m in
// [1, 2)), k = top 7 bits of m, u = m / c_k - 1 (|u| <= 2^-8),
// log x = e ln2 + T_k + log1p(u) with the series to u^5 (the u^6 term is below
// 6e-16). tab[k] = {fl(1/c_k), T_hi, T_lo, 0}, c_k = 1 + (k + 1/2)/128,
// T = -log(fl(1/c_k)) (T_hi rounded to 19 fractional bits, so that
// e ln2_hi + T_hi is exact for |e| <= 15). Integer work is kept to bit
// masks: the table offset, the mantissa, 2^-e and e come straight from the bits.
__device__ __forceinline__ void log_pair_fast(float xh, float xl, const float4* tab, float& S, float& lo)
{
    const int bits = __float_as_int(xh);
    const float4 tk = *(const float4*)((const char*)tab + ((bits >> 12) & 0x7F0));
    const float mh = __int_as_float((bits & 0x007fffff) | 0x3f800000);
    const float ml = __fmul_rn(xl, __int_as_float(0x7F000000 - (bits & 0x7F800000)));  // xl 2^-e
    const float Pm = __fmul_rn(mh, tk.x);
    const float Pe = fmaf(mh, tk.x, -Pm);
    const float uh = __fsub_rn(Pm, 1.0f);
    const float ul = fmaf(ml, tk.x, Pe);
    const float ef = __fsub_rn(__int_as_float((bits >> 23) + (0x4B400000 - 127)), 12582912.0f);  // e
    const float hi = fmaf(ef, kLn2Hi, tk.y);
    const float uhh = __fsub_rn(__fadd_rn(uh, 24.0f), 24.0f);
    const float uhl = __fsub_rn(uh, uhh);
    S = __fadd_rn(hi, uhh);
    const float s2 = __fmul_rn(uh, uh);
    const float s2e = fmaf(uh, uh, -s2);
    const float poly = fmaf(uh, fmaf(uh, 0.2f, -0.25f), 1.0f / 3.0f);
    float tt = __fmul_rn(__fmul_rn(s2, uh), poly);
    tt = fmaf(-uh, ul, tt);
    tt = fmaf(-0.5f, s2e, tt);
    tt = __fadd_rn(tt, ul);
    tt = __fadd_rn(tt, tk.z);
    tt = __fadd_rn(tt, uhl);
    tt = fmaf(-0.5f, s2, tt);
    lo = fmaf(ef, kLn2Lo, tt);
}

// log(x) for any x = xh + xl > 0: the table path for 2^-15 <= xh < 2^16, an
// FP64 log otherwise.
__device__ __forceinline__ void log_pair(float xh, float xl, const float4* tab, float& S, float& lo)
{
    if (xh >= 0x1p-15f && xh < 0x1p16f) {
        log_pair_fast(xh, xl, tab, S, lo);
    } else {
        const double ld = log((double)xh + (double)xl);
        S = __double2float_rn(ld);
        lo = __double2float_rn(ld - (double)S);
    }
}

// 1 / x for x = (xh, xl) > 0: float reciprocal refined by one Newton step in
// float-float (relative error about 2^-46).
__device__ __forceinline__ F recip(F x)
{
    const float r0 = __frcp_rn(x.h);
    float e = fmaf(-x.h, r0, 1.0f);  // exact residual of the hi part
    e = fmaf(-x.l, r0, e);
    return F{r0, __fmul_rn(r0, e)};
}

// (offset + scale * (rh + rl)) for an exact float offset and a power-of-two scale
__device__ __forceinline__ F shift_scale(float off, float scale, float rh, float rl)
{
    float s, e;
    two_sum(off, __fmul_rn(scale, rh), s, e);
    return F{s, __fadd_rn(e, __fmul_rn(scale, rl))};
}

}  // namespace ff
}  // namespace vp
