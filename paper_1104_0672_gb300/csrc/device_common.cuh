// Device helpers shared by the library's kernels (FP64 profile lookup, complex math).
#pragma once

#include <cuda_runtime.h>

#include "arkcos_impl.cuh"

namespace arkcos {

__device__ __forceinline__ float2 cmulf(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 caddf(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csubf(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cconjf(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscalef(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// exp(i pi a / b) for integers with |a| < 2^31 and 0 < b < 2^29: the angle is reduced
// exactly modulo 2b in integer arithmetic, so the FP32 argument lies in [0, 2).
__device__ __forceinline__ float2 expipi_ratio(int a, int b)
{
    int r = a % (2 * b);
    if (r < 0) r += 2 * b;
    float s, c;
    sincospif(__fdiv_rn((float)r, (float)b), &s, &c);
    return make_float2(c, s);
}

// Knot segment t0 with ut[t0] <= u < ut[t0+1] (u already clamped to [0, umax]).
// First guess from the FP32 angle, then exact FP64 comparisons.
__device__ __forceinline__ int knot_segment(double u, const double *ut, int T, double gscale)
{
    float g = 2.0f * asinf(fminf(1.0f, 0.5f * sqrtf((float)u)));
    int t0 = (int)(g * (float)gscale);
    t0 = max(0, min(T - 2, t0));
    while (t0 > 0 && u < ut[t0]) --t0;
    while (t0 < T - 2 && u >= ut[t0 + 1]) ++t0;
    return t0;
}

// Profile value K(u) (linear in u between knots); callers guarantee u <= umax.
__device__ __forceinline__ double profile_eval(double u, const double *ut, const double *f, int T,
                                               double gscale)
{
    int t0 = knot_segment(u, ut, T, gscale);
    double lam = (u - ut[t0]) / (ut[t0 + 1] - ut[t0]);
    return f[t0] + lam * (f[t0 + 1] - f[t0]);
}

}  // namespace arkcos
