// Per-ring helpers shared by the forward and inverse ring transforms (Sec. 4.1).
//
// One CTA owns one ring pair (j, R-1-j): mirror rings have the same length and offset, so
// their two real rings are packed as the real and imaginary parts of one complex sequence
// and split afterwards by Hermitian symmetry.  The CTA loops over all maps of the batch.
// Transforms run in shared memory over a power-of-two buffer M (fft_engine.cuh):
//   - power-of-two rings (M = n): one forward DIF transform (digit-reversed spectrum) or,
//     on the inverse side, the adjoint transform from digit-reversed input;
//   - other lengths: Bluestein's chirp-z algorithm (1970) with M >= 2n - 1: DIF of the
//     chirped sequence, pointwise product with the chirp spectrum (precomputed per grid)
//     fused with the last DIF and first adjoint pass, adjoint back to natural order.
// The buffer size is a compile-time parameter of the per-ring code: a launch covers rings
// of one or several sizes and each CTA branches once to the code for its own size.
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

// Per-CTA tables of a ring of n pixels: chirp[k] = exp(sgn i pi k^2 / n) for k <= n/2
// (Bluestein rings) and phase[m] = exp(sgn i pi m / n) for m <= n/2 (rings with a half-pixel
// offset).
__device__ __forceinline__ void tables(float2 *chirp, float2 *phase, int n, bool blu, bool hs, int sgn)
{
    if (blu)
        for (int k = threadIdx.x; 2 * k <= n; k += blockDim.x) chirp[k] = expipi_ratio(sgn * k * k, n);
    if (hs)
        for (int m = threadIdx.x; m <= n / 2; m += blockDim.x) phase[m] = expipi_ratio(sgn * m, n);
    __syncthreads();
}

// Buffer size of a ring: n itself when it is a power of two, else the Bluestein size.
__device__ __forceinline__ int log2_buffer(int n)
{
    int l = 1;
    while ((1 << l) < n) ++l;
    if ((1 << l) == n) return l;
    l = 1;
    while ((1 << l) < 2 * n - 1) ++l;
    return l;
}

// Calls f.template run<L>() for the runtime buffer size 2^logM (1 <= logM <= 14).
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
    case 13: f.template run<13>(); break;
    default: f.template run<14>(); break;
    }
}

}  // namespace ring
}  // namespace arkcos
