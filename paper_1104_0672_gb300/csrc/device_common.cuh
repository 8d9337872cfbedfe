// Device helpers shared by the library's kernels (FP64 profile lookup, complex math).
#pragma once

#include <cuda_runtime.h>

#include "arkcos_impl.cuh"

namespace arkcos {

__device__ __forceinline__ float2 cmulf(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// complex add and subtract as one packed two-lane FP32 instruction each (same rounding as
// two scalar operations)
__device__ __forceinline__ float2 caddf(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csubf(float2 a, float2 b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(*reinterpret_cast<unsigned long long *>(&a)),
        "l"(*reinterpret_cast<unsigned long long *>(&b)));
    return *reinterpret_cast<float2 *>(&r);
}
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

// The same search in FP32 (knots utf in FP32): next to a knot it may return the neighbouring
// segment, which callers that evaluate a continuous piecewise-linear profile may accept.
__device__ __forceinline__ int knot_segment_f(float u, const float *utf, int T, double gscale)
{
    float g = 2.0f * asinf(fminf(1.0f, 0.5f * sqrtf(u)));
    int t0 = (int)(g * (float)gscale);
    t0 = max(0, min(T - 2, t0));
    while (t0 > 0 && u < utf[t0]) --t0;
    while (t0 < T - 2 && u >= utf[t0 + 1]) ++t0;
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

// rho_m = sum_k tap_k cos((2k + f) alpha), alpha = pi m / N, over k = 0..S.
// Reinsch's recurrence: for cos(2 alpha) >= 0 the difference D_k = C_k - C_{k-1} obeys
// D_{k+1} = D_k - lam C_k (lam = 4 sin^2 alpha); otherwise the sum E_k = C_k + C_{k-1}
// obeys E_{k+1} = mu C_k - E_k (mu = 4 cos^2 alpha).  Rounding error grows linearly in k;
// the state is re-seeded from exact values every 64 taps.
#define REC_STEP()                 \
    do {                           \
        if (low) {                 \
            G = fmaf(-lam, C, G);  \
            C += G;                \
        } else {                   \
            G = fmaf(mu, C, -G);   \
            C = G - C;             \
        }                          \
    } while (0)

__device__ __forceinline__ float gen_rho(const float4 *__restrict__ tp4, int S, int f, int m, int N)
{
    if (S < 0) return 0.f;
    float sa, ca;
    sincospif((float)m / (float)N, &sa, &ca);
    const bool low = (4 * m <= N);
    const float lam = 4.f * sa * sa, mu = 4.f * ca * ca;
    float C = f ? ca : 1.0f;
    float G;  // D_0 (low) or E_0 (high)
    if (low) G = f ? 0.f : 0.5f * lam;
    else G = f ? 2.f * ca : 0.5f * mu;
    float acc = 0.f;
    const int nq = (S + 4) >> 2;
    for (int q = 0; q < nq; ++q) {
        const float4 t4 = __ldg(&tp4[q]);
        if (q > 0) {
            if ((q & 15) == 0) {
                // exact C_k at k = 4q and its recurrence partner (angles (2k+f) alpha and
                // (2k-1+f) alpha, reduced exactly modulo 2N)
                const int k = 4 * q;
                const float2 e1 = expipi_ratio((2 * k + f) * m, N);
                const float2 e2 = expipi_ratio((2 * k - 1 + f) * m, N);
                C = e1.x;
                G = low ? -2.f * e2.y * sa : 2.f * e2.x * ca;
            } else {
                REC_STEP();
            }
        }
        acc = fmaf(t4.x, C, acc);
        REC_STEP();
        acc = fmaf(t4.y, C, acc);
        REC_STEP();
        acc = fmaf(t4.z, C, acc);
        REC_STEP();
        acc = fmaf(t4.w, C, acc);
    }
    return acc;
}

// 16-byte asynchronous global -> shared copy (zero-filled when bytes == 0).
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc, int bytes)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gsrc), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Issue the copies of one map's union band [ju0, ju0 + nu) x `modes` modes starting at mode
// m0 into shared memory, raw paired rows (rows of southern rings keep the stored order).
__device__ __forceinline__ void stage_band_async(float4 *dst, const float4 *__restrict__ sp4b, int ju0,
                                                 int nu, int m0, int modes, int R, int NH)
{
    for (int e = threadIdx.x; e < nu * modes; e += blockDim.x) {
        const int jj = e / modes, mm = m0 + (e - jj * modes);
        const int j = ju0 + jj, jm = R - 1 - j;
        const int rep = j > jm ? jm : j;
        const bool in = mm < NH;
        cp_async16(&dst[e], sp4b + (int64_t)rep * NH + (in ? mm : 0), in ? 16 : 0);
    }
    cp_async_commit();
}

}  // namespace arkcos
