// Power-of-two complex FFT engine for one CTA over a shared-memory buffer (used by the ring
// transforms of Sec. 4.1).
//
// Cooley-Tukey with radix 16 passes (the last pass takes the remaining 1-3 bits):
//   decimation in frequency (DIF), pass over blocks of B = R S: for each block and n2 < S the
//   R elements x[n1 S + n2] go through an R-point DFT held in registers, then output k1 is
//   multiplied by W_B^{n2 k1} (W_B = exp(-2 pi i / B)) and written back in place.  After all
//   passes frequency f sits at digitrev(f): the base-16 digits of f in reverse order.
//   The adjoint passes (conjugate twiddles, then the inverse-sign R-point DFT, in reverse pass
//   order) take a digit-reversed spectrum back to natural order and compute M times the
//   inverse DFT.
// The R-point DFTs split 16 = 4 x 4 and 8 = 4 x 2 with constant internal roots.  Element p
// of a 2^L buffer lives at sp(p) = p + p / 16 + p / 2^(L-4) (the last term for L >= 8): one
// pad slot per 16 elements keeps the radix passes free of shared-memory bank conflicts for
// 8-byte elements, and the top-digit term does the same for reads in digit-reversed order.
#pragma once
#include "device_common.cuh"

namespace arkcos {
namespace fft {

// shift of the top-digit term for a 2^logM buffer (31: no term)
__device__ __forceinline__ int top_shift(int logM) { return logM >= 8 ? logM - 4 : 31; }
__device__ __forceinline__ int sp(int p, int tsh) { return p + (p >> 4) + (p >> tsh); }

// buffer words (float2) for a transform of M points
__host__ __device__ constexpr int buffer_words(int M) { return M + M / 16 + 16; }

// base-16 digit reversal of f over logM bits (the last digit takes the remaining bits)
__device__ __forceinline__ int digitrev(int f, int logM)
{
    int p = 0, left = logM;
    while (left > 0) {
        const int rb = left >= 4 ? 4 : left;
        left -= rb;
        p |= (f & ((1 << rb) - 1)) << left;
        f >>= rb;
    }
    return p;
}

__host__ __device__ constexpr float cos16(int j)
{
    constexpr float C1 = 0.92387953251128674f, S1 = 0.38268343236508978f, H = 0.70710678118654752f;
    switch (j & 15) {
    case 0: return 1.f;   case 1: return C1;   case 2: return H;    case 3: return S1;
    case 4: return 0.f;   case 5: return -S1;  case 6: return -H;   case 7: return -C1;
    case 8: return -1.f;  case 9: return -C1;  case 10: return -H;  case 11: return -S1;
    case 12: return 0.f;  case 13: return S1;  case 14: return H;   default: return C1;
    }
}
__host__ __device__ constexpr float sin16(int j) { return cos16(j - 4); }  // sin(x) = cos(x - pi/2)

// a * W16^J, W16 = exp(-2 pi i / 16); the conjugate root when INV
template <int J, bool INV>
__device__ __forceinline__ float2 rot16(float2 a)
{
    constexpr int j = J & 15;
    if constexpr (j == 0) {
        return a;
    } else if constexpr (j == 4) {
        return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
    } else if constexpr (j == 8) {
        return make_float2(-a.x, -a.y);
    } else if constexpr (j == 12) {
        return INV ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
    } else {
        constexpr float c = cos16(j), s = sin16(j);
        constexpr float si = INV ? s : -s;  // imaginary part of the root
        return make_float2(fmaf(a.x, c, -a.y * si), fmaf(a.x, si, a.y * c));
    }
}

template <bool INV>
__device__ __forceinline__ void dft2(float2 &a, float2 &b)
{
    const float2 s = caddf(a, b), d = csubf(a, b);
    a = s;
    b = d;
}

template <bool INV>
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3)
{
    const float2 t0 = caddf(a0, a2), t1 = csubf(a0, a2), t2 = caddf(a1, a3), t3 = csubf(a1, a3);
    a0 = caddf(t0, t2);
    a2 = csubf(t0, t2);
    if (INV) {  // t1 +- i t3
        a1 = make_float2(t1.x - t3.y, t1.y + t3.x);
        a3 = make_float2(t1.x + t3.y, t1.y - t3.x);
    } else {    // t1 -+ i t3
        a1 = make_float2(t1.x + t3.y, t1.y - t3.x);
        a3 = make_float2(t1.x - t3.y, t1.y + t3.x);
    }
}

// 8 = 4 x 2: n = 2 na + nb, k = ka + 4 kb
template <bool INV>
__device__ __forceinline__ void dft8(float2 (&v)[8])
{
    dft4<INV>(v[0], v[2], v[4], v[6]);
    dft4<INV>(v[1], v[3], v[5], v[7]);
    // v[2 ka + nb] holds t[nb][ka]
    v[3] = rot16<2, INV>(v[3]);
    v[5] = rot16<4, INV>(v[5]);
    v[7] = rot16<6, INV>(v[7]);
    float2 o[8];
    o[0] = caddf(v[0], v[1]); o[4] = csubf(v[0], v[1]);
    o[1] = caddf(v[2], v[3]); o[5] = csubf(v[2], v[3]);
    o[2] = caddf(v[4], v[5]); o[6] = csubf(v[4], v[5]);
    o[3] = caddf(v[6], v[7]); o[7] = csubf(v[6], v[7]);
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = o[k];
}

// 16 = 4 x 4: n = 4 na + nb, k = ka + 4 kb
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&v)[16])
{
#pragma unroll
    for (int nb = 0; nb < 4; ++nb) dft4<INV>(v[nb], v[4 + nb], v[8 + nb], v[12 + nb]);
    // v[4 ka + nb] holds t[nb][ka]; multiply by W16^{nb ka}
    v[5] = rot16<1, INV>(v[5]);
    v[6] = rot16<2, INV>(v[6]);
    v[7] = rot16<3, INV>(v[7]);
    v[9] = rot16<2, INV>(v[9]);
    v[10] = rot16<4, INV>(v[10]);
    v[11] = rot16<6, INV>(v[11]);
    v[13] = rot16<3, INV>(v[13]);
    v[14] = rot16<6, INV>(v[14]);
    v[15] = rot16<9, INV>(v[15]);
#pragma unroll
    for (int ka = 0; ka < 4; ++ka) dft4<INV>(v[4 * ka], v[4 * ka + 1], v[4 * ka + 2], v[4 * ka + 3]);
    // v[4 ka + kb] holds X[ka + 4 kb]: transpose the 4 x 4 index
    float2 o[16];
#pragma unroll
    for (int ka = 0; ka < 4; ++ka)
#pragma unroll
        for (int kb = 0; kb < 4; ++kb) o[ka + 4 * kb] = v[4 * ka + kb];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = o[k];
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2 (&v)[R])
{
    if constexpr (R == 16) dft16<INV>(v);
    else if constexpr (R == 8) dft8<INV>(v);
    else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 2) dft2<INV>(v[0], v[1]);
}

// v[k] *= W_B^{n2 k} (conjugated when CONJ) for k = 1..R-1, n2 < B / R.  tw[h + p] holds
// exp(-2 pi i p / (2h)) for p < h; the products n2 k read from the table stay below B / 2.
template <int R, bool CONJ>
__device__ __forceinline__ void twiddle(float2 (&v)[R], const float2 *__restrict__ tw, int B, int n2)
{
    const float2 *t = tw + (B >> 1);
    auto ld = [&](int j) {
        float2 w = __ldg(&t[j]);
        if (CONJ) w.y = -w.y;
        return w;
    };
    if constexpr (R == 2) {
        v[1] = cmulf(v[1], ld(n2));
    } else if constexpr (R == 4) {
        const float2 w1 = ld(n2), w2 = ld(2 * n2);
        v[1] = cmulf(v[1], w1);
        v[2] = cmulf(v[2], w2);
        v[3] = cmulf(v[3], cmulf(w1, w2));
    } else {
        // w^{4a + b} = w^{4a} w^b with w^1..w^4 from the table, applied as generated
        const float2 w1 = ld(n2), w2 = ld(2 * n2), w3 = ld(3 * n2), w4 = ld(4 * n2);
        v[1] = cmulf(v[1], w1);
        v[2] = cmulf(v[2], w2);
        v[3] = cmulf(v[3], w3);
        float2 wa = w4;
#pragma unroll
        for (int a = 4; a < R; a += 4) {
            if (a > 4) wa = cmulf(wa, w4);
            v[a] = cmulf(v[a], wa);
            v[a + 1] = cmulf(v[a + 1], cmulf(wa, w1));
            v[a + 2] = cmulf(v[a + 2], cmulf(wa, w2));
            v[a + 3] = cmulf(v[a + 3], cmulf(wa, w3));
        }
    }
}

// Shared-memory element access of a buffer with top-digit shift tsh.
struct Smem {
    float2 *x;
    int tsh;
    __device__ __forceinline__ float2 operator()(int p) const { return x[sp(p, tsh)]; }
    __device__ __forceinline__ void operator()(int p, float2 v) const { x[sp(p, tsh)] = v; }
    // sp(base + r S) = sp(base) + r stride(S) for S >= 16 (S a multiple of 16, and the top
    // digit either constant over the block or equal to r when S is the top stride)
    __device__ __forceinline__ int stride(int S) const { return S + (S >> 4) + (S == (1 << tsh) ? 1 : 0); }
};

template <class T> struct is_smem { static constexpr bool value = false; };
template <> struct is_smem<Smem> { static constexpr bool value = true; };

// One pass over blocks of R * S points.  DIF (ADJ false): R-point DFT, then twiddles.
// Adjoint (ADJ true): conjugate twiddles, then the inverse-sign R-point DFT.  Elements are
// read through ld(p) and written through st(p, v) (shared memory, or the first/last pass
// fused with global input/output).
template <int R, bool ADJ, class Ld, class St>
__device__ __forceinline__ void pass(int M, int S, const float2 *__restrict__ tw, Ld ld, St st)
{
    const int groups = M / R;
    for (int g = threadIdx.x; g < groups; g += blockDim.x) {
        const int n2 = g & (S - 1);
        const int base = (g - n2) * R + n2;
        float2 v[R];
        if constexpr (is_smem<Ld>::value) {
            if (S >= 16) {
                const int a0 = sp(base, ld.tsh), as = ld.stride(S);
#pragma unroll
                for (int r = 0; r < R; ++r) v[r] = ld.x[a0 + r * as];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) v[r] = ld(base + r * S);
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = ld(base + r * S);
        }
        if (!ADJ) {
            dft<R, false>(v);
            if (S > 1) twiddle<R, false>(v, tw, R * S, n2);
        } else {
            if (S > 1) twiddle<R, true>(v, tw, R * S, n2);
            dft<R, true>(v);
        }
        if constexpr (is_smem<St>::value) {
            if (S >= 16) {
                const int a0 = sp(base, st.tsh), as = st.stride(S);
#pragma unroll
                for (int r = 0; r < R; ++r) st.x[a0 + r * as] = v[r];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) st(base + r * S, v[r]);
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) st(base + r * S, v[r]);
        }
    }
    __syncthreads();
}

template <bool ADJ, class Ld, class St>
__device__ __forceinline__ void pass_bits(int rb, int M, int S, const float2 *__restrict__ tw, Ld ld, St st)
{
    switch (rb) {
    case 4: pass<16, ADJ>(M, S, tw, ld, st); break;
    case 3: pass<8, ADJ>(M, S, tw, ld, st); break;
    case 2: pass<4, ADJ>(M, S, tw, ld, st); break;
    default: pass<2, ADJ>(M, S, tw, ld, st); break;
    }
}

// radix bits of the last DIF pass (= first adjoint pass)
__device__ __forceinline__ int last_bits(int logM) { return (logM & 3) ? (logM & 3) : 4; }

// Forward DIF over M = 2^logM into the buffer x: natural-order input read through ld(k) by
// the first pass, digit-reversed spectrum out.  With skip_last the final pass (blocks of
// 2^last_bits, no twiddles) is left to the caller.
template <class Ld>
__device__ __forceinline__ void dif(float2 *x, int logM, const float2 *__restrict__ tw, Ld ld,
                                    bool skip_last = false)
{
    const int M = 1 << logM;
    const Smem sm{x, top_shift(logM)};
    if (skip_last && logM <= 4) {  // a single pass, left to the caller: just stage the input
        for (int k = threadIdx.x; k < M; k += blockDim.x) sm(k, ld(k));
        __syncthreads();
        return;
    }
    int S = M, left = logM;
    bool first = true;
    while (left > 0) {
        const int rb = left >= 4 ? 4 : left;
        S >>= rb;
        if (skip_last && left == rb) break;
        if (first) pass_bits<false>(rb, M, S, tw, ld, sm);
        else pass_bits<false>(rb, M, S, tw, sm, sm);
        first = false;
        left -= rb;
    }
}

// Adjoint of dif: digit-reversed spectrum in x, M x inverse DFT out in natural order,
// written through st(k, v) by the last pass.  With skip_first the first pass is taken to be
// done already.
template <class St>
__device__ __forceinline__ void adj(float2 *x, int logM, const float2 *__restrict__ tw, St st,
                                    bool skip_first = false)
{
    const int M = 1 << logM;
    const Smem sm{x, top_shift(logM)};
    int S = 1, done = 0;
    while (done < logM) {
        const int rb = done == 0 ? last_bits(logM) : 4;
        const bool last = done + rb == logM;
        if (skip_first && done == 0) {
            if (last) {  // a single pass, done by the caller: just write the output
                for (int k = threadIdx.x; k < M; k += blockDim.x) st(k, sm(k));
                __syncthreads();
            }
        } else if (last) {
            pass_bits<true>(rb, M, S, tw, sm, st);
        } else {
            pass_bits<true>(rb, M, S, tw, sm, sm);
        }
        S <<= rb;
        done += rb;
    }
}

// The last DIF pass, the pointwise product with the spectrum fb (digit-reversed positions,
// conjugated when CONJ) and the first adjoint pass, fused: blocks of R points, no twiddles.
template <int R, bool CONJ>
__device__ __forceinline__ void middle(const Smem &sm, int M, const float2 *__restrict__ fb)
{
    const int groups = M / R;
    for (int g = threadIdx.x; g < groups; g += blockDim.x) {
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = sm(g * R + r);
        dft<R, false>(v);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 f = __ldg(&fb[g * R + r]);
            if (CONJ) f.y = -f.y;
            v[r] = cmulf(v[r], f);
        }
        dft<R, true>(v);
#pragma unroll
        for (int r = 0; r < R; ++r) sm(g * R + r, v[r]);
    }
    __syncthreads();
}

// M times the circular convolution of the input (natural order, read through ld) with the
// sequence whose DIF spectrum fb holds (digit-reversed positions; conjugated when CONJ).
// The result, in natural order, is written through st.
template <bool CONJ, class Ld, class St>
__device__ __forceinline__ void convolve(float2 *x, int logM, const float2 *__restrict__ tw,
                                         const float2 *__restrict__ fb, Ld ld, St st)
{
    const int M = 1 << logM;
    const Smem sm{x, top_shift(logM)};
    dif(x, logM, tw, ld, true);
    switch (last_bits(logM)) {
    case 4: middle<16, CONJ>(sm, M, fb); break;
    case 3: middle<8, CONJ>(sm, M, fb); break;
    case 2: middle<4, CONJ>(sm, M, fb); break;
    default: middle<2, CONJ>(sm, M, fb); break;
    }
    adj(x, logM, tw, st, true);
}

}  // namespace fft
}  // namespace arkcos
