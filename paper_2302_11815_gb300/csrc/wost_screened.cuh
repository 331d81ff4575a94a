// Screened Poisson equation (App. A.2) on the device: scaled modified
// Bessel functions, the Green's function of the ball and the step weight Q.
// Included by the screened translation unit only.
#pragma once

#include "wost_device.cuh"

namespace wost {

// ---------------------------------------------------------------------------
// screened Poisson equation (App. A.2)
// ---------------------------------------------------------------------------
// Exponentially scaled modified Bessel functions e^-x I0, e^-x I1, e^x K0,
// e^x K1 (x > 0) by the polynomial approximations of Abramowitz & Stegun,
// Handbook of Mathematical Functions, 9.8.1-9.8.8 (absolute/relative error
// below 2.2e-7 in the scaled forms).
__device__ __forceinline__ float poly(float t, const float *c, int n) {
    float r = c[n - 1];
    for (int i = n - 2; i >= 0; --i) r = fmaf(r, t, c[i]);
    return r;
}
static __device__ __noinline__ float bessel_i0e(float x) {
    if (x <= 3.75f) {
        const float c[7] = {1.f, 3.5156229f, 3.0899424f, 1.2067492f, 0.2659732f, 0.0360768f, 0.0045813f};
        float t = x * (1.f / 3.75f);
        return poly(t * t, c, 7) * expf(-x);
    }
    const float c[9] = {0.39894228f, 0.01328592f, 0.00225319f, -0.00157565f, 0.00916281f,
                        -0.02057706f, 0.02635537f, -0.01647633f, 0.00392377f};
    return poly(3.75f / x, c, 9) * rsqrtf(x);
}
static __device__ __noinline__ float bessel_i1e(float x) {
    if (x <= 3.75f) {
        const float c[7] = {0.5f, 0.87890594f, 0.51498869f, 0.15084934f, 0.02658733f, 0.00301532f, 0.00032411f};
        float t = x * (1.f / 3.75f);
        return x * poly(t * t, c, 7) * expf(-x);
    }
    const float c[9] = {0.39894228f, -0.03988024f, -0.00362018f, 0.00163801f, -0.01031555f,
                        0.02282967f, -0.02895312f, 0.01787654f, -0.00420059f};
    return poly(3.75f / x, c, 9) * rsqrtf(x);
}
static __device__ __noinline__ float bessel_k0e(float x) {
    if (x <= 2.f) {
        const float c[7] = {-0.57721566f, 0.42278420f, 0.23069756f, 0.03488590f, 0.00262698f, 0.00010750f,
                            0.00000740f};
        float h = 0.5f * x;
        return (-logf(h) * bessel_i0e(x) * expf(x) + poly(h * h, c, 7)) * expf(x);
    }
    const float c[7] = {1.25331414f, -0.07832358f, 0.02189568f, -0.01062446f, 0.00587872f, -0.00251540f,
                        0.00053208f};
    return poly(2.f / x, c, 7) * rsqrtf(x);
}
static __device__ __noinline__ float bessel_k1e(float x) {
    if (x <= 2.f) {
        const float c[7] = {1.f, 0.15443144f, -0.67278579f, -0.18156897f, -0.01919402f, -0.00110404f,
                            -0.00004686f};
        float h = 0.5f * x;
        return (x * logf(h) * bessel_i1e(x) * expf(x) + poly(h * h, c, 7)) / x * expf(x);
    }
    const float c[7] = {1.25331414f, 0.23498619f, -0.03655620f, 0.01504268f, -0.00780353f, 0.00325614f,
                        -0.00068245f};
    return poly(2.f / x, c, 7) * rsqrtf(x);
}

// Green's function of the ball B(x,R) at distance rho (Eq.
// GreensFnsScreenedPoissonBall), sqs = sqrt(sigma); written with the scaled
// Bessel functions and exponentials so that nothing overflows.
template <int D>
__device__ __noinline__ float screened_green(float rho, float R, float sqs) {
    const float a = R * sqs, b = rho * sqs;
    if constexpr (D == 2) {
        float k0b = bessel_k0e(b) * expf(-b);
        float ratio = bessel_i0e(b) * bessel_k0e(a) / bessel_i0e(a) * expf(b - 2.f * a);
        return (k0b - ratio) * (0.5f / 3.14159265358979f);
    } else {
        // sinh((R - rho) s) / sinh(R s)
        float ratio = expf(-b) * expm1f(-2.f * (a - b)) / expm1f(-2.f * a);
        return ratio / (4.f * 3.14159265358979f * rho);
    }
}
// step weight Q^sigma_B at distance rho <= R (Eq. ScreenedPoissonKernelsSphere)
template <int D>
__device__ __noinline__ float screened_q(float rho, float R, float sqs) {
    const float a = R * sqs, b = rho * sqs;
    if constexpr (D == 2) {
        float k1b = bessel_k1e(b) * expf(-b);
        float ratio = bessel_i1e(b) * bessel_k0e(a) / bessel_i0e(a) * expf(b - 2.f * a);
        return (k1b + ratio) * b;
    } else {
        // (b cosh b - sinh b) e^-a / sinh a; its series b^3/3 (1 + b^2/10 +
        // b^4/280) for small b, where the exponentials cancel
        float denom = -expm1f(-2.f * a);
        float second;
        if (b < 0.1f) {
            float b2 = b * b;
            second = (b2 * b * (1.f / 3.f)) * (1.f + b2 * (0.1f + b2 * (1.f / 280.f))) * 2.f * expf(-2.f * a) / denom;
        } else {
            second = ((b - 1.f) * expf(b - 2.f * a) + (b + 1.f) * expf(-b - 2.f * a)) / denom;
        }
        return expf(-b) * (b + 1.f) + second;
    }
}

}  // namespace wost
