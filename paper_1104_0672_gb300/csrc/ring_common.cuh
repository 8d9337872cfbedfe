// Per-ring helpers shared by the forward and inverse ring transforms (Sec. 4.1).
//
// One CTA owns one ring pair (j, R-1-j): mirror rings have the same length n and offset, so
// their transforms share every twiddle.  Each ring (n even) is read as the complex sequence
// z_q = x_2q + i x_2q+1 of h = n/2 points, whose h-point DFT Z gives the ring's half spectrum
// by the split X_k = (Z_k + conj Z_{h-k}) / 2 - i exp(-2 pi i k / n) (Z_k - conj Z_{h-k}) / 2;
// the two rings of the pair are the two lanes of the engine's packed element (fft::cpair).
// The CTA loops over maps.  Transforms run in shared memory over a power-of-two buffer M
// (fft_engine.cuh):
//   - h a power of two (M = h): one forward DIF transform (digit-reversed spectrum) or, on the
//     inverse side, the adjoint transform from digit-reversed input;
//   - other h: Bluestein's chirp-z algorithm (1970) with M >= 2h - 1: DIF of the chirped
//     sequence, pointwise product with the chirp spectrum (precomputed per grid) fused with
//     the last DIF and first adjoint pass, adjoint back to natural order.
// The buffer size is a compile-time parameter of the per-ring code: a launch covers rings of
// one or several sizes and each CTA branches once to the code for its own size.  Rings too
// long for the largest buffer (n = 4q, 2h - 1 > 8192) go through four q-point transforms
// instead (the split path, one ring pair packed as one complex sequence).
#pragma once
#include "fft_engine.cuh"

namespace arkcos {
namespace ring {

// chirp(k) = exp(sgn i pi k^2 / n) for k < n from the table of k <= n/2:
// chirp(n - k) = (-1)^n chirp(k)
__device__ __forceinline__ float2 chirp_at(const float2 *chirp, int k, int n)
{
    if (2 * k <= n) return chirp[k];
    const float2 c = chirp[n - k];
    return (n & 1) ? make_float2(-c.x, -c.y) : c;
}

// Per-CTA tables of a ring of n pixels: phase[m] = exp(sgn i pi m / n) for m <= n/2 (the
// first-pixel phase of half-pixel rings, and at even m the split twiddles) -- for a
// power-of-two n copied from the stage twiddles (tw[n + m] = exp(-i pi m / n)) -- and, when
// its h-point transform goes by Bluestein, chirp[k] = exp(sgn i pi k^2 / h) for k <= h/2.
__device__ __forceinline__ void tables(float2 *chirp, float2 *phase, int n, int h, int sgn, bool blu,
                                       const float2 *__restrict__ tw)
{
    if (blu) {
        for (int k = threadIdx.x; 2 * k <= h; k += blockDim.x) chirp[k] = expipi_ratio(sgn * k * k, h);
        for (int m = threadIdx.x; 2 * m <= n; m += blockDim.x) phase[m] = expipi_ratio(sgn * m, n);
    } else {
        for (int m = threadIdx.x; 2 * m <= n; m += blockDim.x) {
            const float2 w = __ldg(&tw[n + m]);
            phase[m] = sgn < 0 ? w : make_float2(w.x, -w.y);
        }
    }
    __syncthreads();
}

// Per-CTA chirp table of the split path: chirp[k] = exp(sgn i pi k^2 / q), k <= q/2.
__device__ __forceinline__ void chirp_table(float2 *chirp, int q, int sgn)
{
    for (int k = threadIdx.x; 2 * k <= q; k += blockDim.x) chirp[k] = expipi_ratio(sgn * k * k, q);
    __syncthreads();
}

// Buffer size of an l-point complex transform: l itself when it is a power of two, else the
// Bluestein size (at least 2).
__host__ __device__ __forceinline__ int log2_buffer(int l)
{
    int b = 1;
    while ((1 << b) < l) ++b;
    if ((1 << b) == l) return b;
    b = 1;
    while ((1 << b) < 2 * l - 1) ++b;
    return b;
}

// Whether the h-point transform of a ring goes by Bluestein (h not a power of two, or h = 1,
// which runs as a 2-point buffer).
__host__ __device__ __forceinline__ bool bluestein(int h) { return h < 2 || (h & (h - 1)) != 0; }

// Calls f.template run<L>() for the runtime buffer size 2^logM (1 <= logM <= 13).
template <class F>
__device__ __forceinline__ void dispatch(int logM, F &f)
{
    switch (logM) {
    case 1: f.template run<1>(); break;
    case 2: f.template run<2>(); break;
    case 3: f.template run<3>(); break;
    case 4: f.template run<4>(); break;
    case 5: f.template run<5>(); break;
    case 6: f.template run<6>(); break;
    case 7: f.template run<7>(); break;
    case 8: f.template run<8>(); break;
    case 9: f.template run<9>(); break;
    case 10: f.template run<10>(); break;
    case 11: f.template run<11>(); break;
    case 12: f.template run<12>(); break;
    default: f.template run<13>(); break;
    }
}

// The same for the launch of one buffer class.  The host puts every ring whose buffer is at
// most 2^10 into class 10 and every other ring into the class of exactly its own buffer, so a
// class LMAX >= 11 needs the code of its own size only (the other sizes are not instantiated).
template <int LMAX, class F>
__device__ __forceinline__ void dispatch_upto(int logM, F &f)
{
    if constexpr (LMAX >= 11) {
        (void)logM;
        f.template run<LMAX>();
    } else {
        switch (logM) {
        case 1: f.template run<1>(); break;
        case 2: f.template run<2>(); break;
        case 3: f.template run<3>(); break;
        case 4: f.template run<4>(); break;
        case 5: f.template run<5>(); break;
        case 6: f.template run<6>(); break;
        case 7: f.template run<7>(); break;
        case 8: f.template run<8>(); break;
        case 9: f.template run<9>(); break;
        default: f.template run<10>(); break;
        }
    }
}

// Launch shape of the class of buffers up to 2^LMAX (LMAX >= 10): one thread per radix-16
// group of the largest buffer, at least 256 (the short rings' folds and extensions run over
// all kernel-grid modes with the whole CTA), and two CTAs per SM below the largest buffer, so
// that the register budget follows.
template <int LMAX>
struct ClassShape {
    static constexpr int kThreads = (1 << LMAX) / 16 < 256 ? 256 : (1 << LMAX) / 16;
    static constexpr int kMinBlocks = LMAX >= 13 ? 1 : 2;
};

// Programmatic dependent launch inside one transform stage.  The buffer classes of a stage
// write disjoint rings and read only what earlier stages wrote, so a class kernel lets the
// next class of the stage start as soon as all of its own CTAs are running (they fill the
// SMs its last wave leaves idle), and each CTA waits for the previous class to complete only
// before it exits: a stage still completes in stream order.  Both instructions do nothing in
// a launch without the programmatic-serialization attribute.
__device__ __forceinline__ void stage_allow_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void stage_wait_prev() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Lane views of a packed pair: (re, im) of lane 0 (ring j) and lane 1 (ring R-1-j).
__device__ __forceinline__ float4 lanes4(const fft::cpair &x) { return make_float4(x.re.x, x.im.x, x.re.y, x.im.y); }

}  // namespace ring
}  // namespace arkcos
