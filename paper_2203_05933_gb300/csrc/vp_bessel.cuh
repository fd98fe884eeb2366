// Modified Bessel functions for the modified-Helmholtz kernel
// G(r, r0) = (lambda^2 / 2 pi) K0(lambda |r - r0|) (arXiv 2203.05933, Sec. 2,
// the Green function stated for L = -Delta + lambda^2), in FP64, usable on the
// host (plan-time operator tables) and on the device (kernels).
//
//   h_m(y) = sum_k y^k / (k! (m + k)!),  y = x^2 / 4, so that I_m(x) = (x/2)^m h_m(y).
//            All terms are positive; the series is summed until a term falls
//            below 2^-60 of the sum. h satisfies h_{m-1} = m h_m + y h_{m+1}, the
//            recurrence of I_m, which is stable downwards (I_m is the minimal
//            solution as m grows).
//   K0, K1   for x <= 2 by their ascending series (Abramowitz & Stegun 9.6.13 and
//            9.6.11 with n = 1); for x > 2 by the trapezoidal rule on
//            K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt, written as
//            exp(-x) int exp(-2 x sinh^2(t/2)) cosh(nu t) dt, step
//            min(0.2, 0.6 / sqrt(x)), terms until the integrand is below 1e-18
//            (the rule converges geometrically for this analytic, rapidly decaying
//            integrand; at most 19 terms for x > 2). Relative error about 1e-15.
//   K_n      from K0, K1 by the forward recurrence K_{n+1} = K_{n-1} + (2n/x) K_n,
//            stable upwards (K_n is the dominant solution).
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define VP_HD __host__ __device__ __forceinline__
#else
#define VP_HD inline
#endif

namespace vp {
namespace bessel {

constexpr double kEulerGamma = 0.577215664901532860606512090082402431;

// h_m(y) given inv_mfact = 1/m!
VP_HD double h_series(int m, double y, double inv_mfact)
{
    double t = inv_mfact, s = inv_mfact;
    for (int k = 1; k < 400; ++k) {
        t *= y / ((double)k * (double)(m + k));
        s += t;
        if (t <= s * 0x1p-60) break;
    }
    return s;
}

// h_m(y) and h_{m+1}(y) in one pass (inv_mfact = 1/m!)
VP_HD void h_series2(int m, double y, double inv_mfact, double& hm, double& hm1)
{
    const double inv_m1 = inv_mfact / (double)(m + 1);
    double t = inv_mfact, t1 = inv_m1, s = inv_mfact, s1 = inv_m1;
    for (int k = 1; k < 400; ++k) {
        const double yk = y / (double)k;
        t *= yk / (double)(m + k);
        t1 *= yk / (double)(m + 1 + k);
        s += t;
        s1 += t1;
        if (t <= s * 0x1p-60) break;
    }
    hm = s;
    hm1 = s1;
}

// K0(x), K1(x) for x > 0
VP_HD void k01(double x, double& k0, double& k1)
{
    if (x <= 2.0) {
        const double y = 0.25 * x * x;
        double t0 = 1.0, t1 = 1.0, H = 0.0;
        double i0 = 1.0, s0 = 0.0, i1 = 1.0, s1 = 1.0 - 2.0 * kEulerGamma;  // k = 0 terms
        for (int k = 1; k <= 14; ++k) {
            t0 *= y / ((double)k * (double)k);
            t1 *= y / ((double)k * (double)(k + 1));
            H += 1.0 / (double)k;
            i0 += t0;
            s0 += H * t0;
            i1 += t1;
            // psi(k+1) + psi(k+2) = 2 H_k + 1/(k+1) - 2 gamma
            s1 += (2.0 * H + 1.0 / (double)(k + 1) - 2.0 * kEulerGamma) * t1;
        }
        const double L = log(0.5 * x);
        k0 = -(L + kEulerGamma) * i0 + s0;
        k1 = 1.0 / x + L * (0.5 * x) * i1 - 0.25 * x * s1;
        return;
    }
    const double h = fmin(0.2, 0.6 / sqrt(x));
    double a0 = 0.5, a1 = 0.5;
    for (int k = 1; k < 64; ++k) {
        const double t = h * (double)k;
        const double sh = sinh(0.5 * t);
        const double e = exp(-2.0 * x * sh * sh);
        a0 += e;
        a1 += e * cosh(t);
        if (e < 1e-18) break;
    }
    const double ex = exp(-x) * h;
    k0 = a0 * ex;
    k1 = a1 * ex;
}

// K0(x) alone for x > 2 (the integral representation above)
VP_HD double k0_large(double x)
{
    const double h = fmin(0.2, 0.6 / sqrt(x));
    double a0 = 0.5;
    for (int k = 1; k < 64; ++k) {
        const double sh = sinh(0.5 * h * (double)k);
        const double e = exp(-2.0 * x * sh * sh);
        a0 += e;
        if (e < 1e-18) break;
    }
    return a0 * exp(-x) * h;
}

}  // namespace bessel
}  // namespace vp
