// Power-of-two complex FFT engine for one CTA over a shared-memory buffer (used by the ring
// transforms of Sec. 4.1 and the FFT forms of the polar coefficients and knot projection).
// The transform size M = 2^L is a template parameter, so every stride, shift and loop bound
// below is a compile-time constant.
//
// Cooley-Tukey with radix 16 passes (the last pass takes the remaining 1-3 bits):
//   decimation in frequency (DIF), pass over blocks of B = R S: for each block and n2 < S the
//   R elements x[n1 S + n2] go through an R-point DFT held in registers, then output k1 is
//   multiplied by W_B^{n2 k1} (W_B = exp(-2 pi i / B)) and written back in place.  After all
//   passes frequency f sits at digitrev(f): the base-16 digits of f in reverse order.
//   The adjoint passes (conjugate twiddles, then the inverse-sign R-point DFT, in reverse pass
//   order) take a digit-reversed spectrum back to natural order and compute M times the
//   inverse DFT.
// The R-point DFTs split 16 = 4 x 4 and 8 = 4 x 2 with constant internal roots.
//
// Element types: float2 is one complex value; cpair is two complex values transformed
// together (two sequences with the same twiddles), held as packed two-lane FP32 registers
// re = (Re a, Re b), im = (Im a, Im b), so that one packed instruction does the work of two
// scalar ones and the twiddles, index arithmetic and shared-memory instructions are shared.
//
// Element p of the buffer lives at sp(p) = p + p / 16 + p / 2^(L-4) (the last term for
// L >= 8): one pad element per 16 keeps the radix passes free of shared-memory bank conflicts
// for 8- and 16-byte elements (the last pass of a radix below 16 gives each thread 16
// consecutive elements), and the top-digit term does the same for reads in digit-reversed
// order (checked with a bank model over L <= 13).
#pragma once
#include "device_common.cuh"

namespace arkcos {
namespace fft {

// two complex values as packed lanes
struct cpair {
    float2 re, im;
};

// buffer elements for a transform of M points
__host__ __device__ constexpr int buffer_words(int M) { return M + M / 16 + 16; }

template <int L>
struct Geo {
    static constexpr int M = 1 << L;
    static constexpr int TSH = L >= 8 ? L - 4 : 31;       // shift of the top-digit term
    static constexpr int NP = (L + 3) / 4;                 // passes
    static constexpr int LAST = (L & 3) ? (L & 3) : 4;     // radix bits of the last DIF pass
    __device__ static constexpr int sp(int p) { return p + (p >> 4) + (p >> TSH); }
    // radix bits and stride of DIF pass I
    __host__ __device__ static constexpr int rb(int I) { return I == NP - 1 ? LAST : 4; }
    __host__ __device__ static constexpr int S(int I) { return M >> (4 * I + rb(I)); }
};

// base-16 digit reversal of f over L bits (the last digit takes the remaining bits)
template <int L>
__device__ __forceinline__ int digitrev(int f)
{
    int p = 0;
#pragma unroll
    for (int d = 0; d < Geo<L>::NP; ++d) {
        const int rb = Geo<L>::rb(d);
        const int left = L - 4 * d - rb;
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

// ---------------------------------------------------------------- element operations
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 bcast(float x) { return make_float2(x, x); }

__device__ __forceinline__ float2 e_add(float2 a, float2 b) { return caddf(a, b); }
__device__ __forceinline__ float2 e_sub(float2 a, float2 b) { return csubf(a, b); }
__device__ __forceinline__ float2 e_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 e_addmi(float2 a, float2 b) { return make_float2(a.x + b.y, a.y - b.x); }  // a - i b
__device__ __forceinline__ float2 e_addpi(float2 a, float2 b) { return make_float2(a.x - b.y, a.y + b.x); }  // a + i b
__device__ __forceinline__ float2 e_mulmi(float2 a) { return make_float2(a.y, -a.x); }  // -i a
__device__ __forceinline__ float2 e_mulpi(float2 a) { return make_float2(-a.y, a.x); }  // +i a
__device__ __forceinline__ float2 e_mul(float2 a, float2 w) { return cmulf(a, w); }
__device__ __forceinline__ float2 e_zero(float2) { return make_float2(0.f, 0.f); }

__device__ __forceinline__ cpair e_add(cpair a, cpair b) { return cpair{caddf(a.re, b.re), caddf(a.im, b.im)}; }
__device__ __forceinline__ cpair e_sub(cpair a, cpair b) { return cpair{csubf(a.re, b.re), csubf(a.im, b.im)}; }
__device__ __forceinline__ cpair e_neg(cpair a) { return cpair{pmul(a.re, bcast(-1.f)), pmul(a.im, bcast(-1.f))}; }
__device__ __forceinline__ cpair e_addmi(cpair a, cpair b) { return cpair{caddf(a.re, b.im), csubf(a.im, b.re)}; }
__device__ __forceinline__ cpair e_addpi(cpair a, cpair b) { return cpair{csubf(a.re, b.im), caddf(a.im, b.re)}; }
__device__ __forceinline__ cpair e_mulmi(cpair a) { return cpair{a.im, pmul(a.re, bcast(-1.f))}; }
__device__ __forceinline__ cpair e_mulpi(cpair a) { return cpair{pmul(a.im, bcast(-1.f)), a.re}; }
// both lanes times the complex scalar w
__device__ __forceinline__ cpair e_mul(cpair a, float2 w)
{
    return cpair{pfma(a.im, bcast(-w.y), pmul(a.re, bcast(w.x))), pfma(a.im, bcast(w.x), pmul(a.re, bcast(w.y)))};
}
__device__ __forceinline__ cpair e_zero(cpair) { return cpair{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }

// a * W16^J, W16 = exp(-2 pi i / 16); the conjugate root when INV
template <int J, bool INV, class E>
__device__ __forceinline__ E rot16(E a)
{
    constexpr int j = J & 15;
    if constexpr (j == 0) {
        return a;
    } else if constexpr (j == 4) {
        return INV ? e_mulpi(a) : e_mulmi(a);
    } else if constexpr (j == 8) {
        return e_neg(a);
    } else if constexpr (j == 12) {
        return INV ? e_mulmi(a) : e_mulpi(a);
    } else {
        constexpr float c = cos16(j), s = sin16(j);
        constexpr float si = INV ? s : -s;  // imaginary part of the root
        return e_mul(a, make_float2(c, si));
    }
}

template <bool INV, class E>
__device__ __forceinline__ void dft2(E &a, E &b)
{
    const E s = e_add(a, b), d = e_sub(a, b);
    a = s;
    b = d;
}

template <bool INV, class E>
__device__ __forceinline__ void dft4(E &a0, E &a1, E &a2, E &a3)
{
    const E t0 = e_add(a0, a2), t1 = e_sub(a0, a2), t2 = e_add(a1, a3), t3 = e_sub(a1, a3);
    a0 = e_add(t0, t2);
    a2 = e_sub(t0, t2);
    if (INV) {  // t1 +- i t3
        a1 = e_addpi(t1, t3);
        a3 = e_addmi(t1, t3);
    } else {    // t1 -+ i t3
        a1 = e_addmi(t1, t3);
        a3 = e_addpi(t1, t3);
    }
}

// 8 = 4 x 2: n = 2 na + nb, k = ka + 4 kb
template <bool INV, class E>
__device__ __forceinline__ void dft8(E (&v)[8])
{
    dft4<INV>(v[0], v[2], v[4], v[6]);
    dft4<INV>(v[1], v[3], v[5], v[7]);
    // v[2 ka + nb] holds t[nb][ka]
    v[3] = rot16<2, INV>(v[3]);
    v[5] = rot16<4, INV>(v[5]);
    v[7] = rot16<6, INV>(v[7]);
    E o[8];
    o[0] = e_add(v[0], v[1]); o[4] = e_sub(v[0], v[1]);
    o[1] = e_add(v[2], v[3]); o[5] = e_sub(v[2], v[3]);
    o[2] = e_add(v[4], v[5]); o[6] = e_sub(v[4], v[5]);
    o[3] = e_add(v[6], v[7]); o[7] = e_sub(v[6], v[7]);
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = o[k];
}

// 16 = 4 x 4: n = 4 na + nb, k = ka + 4 kb
template <bool INV, class E>
__device__ __forceinline__ void dft16(E (&v)[16])
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
    E o[16];
#pragma unroll
    for (int ka = 0; ka < 4; ++ka)
#pragma unroll
        for (int kb = 0; kb < 4; ++kb) o[ka + 4 * kb] = v[4 * ka + kb];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = o[k];
}

template <int R, bool INV, class E>
__device__ __forceinline__ void dft(E (&v)[R])
{
    if constexpr (R == 16) dft16<INV>(v);
    else if constexpr (R == 8) dft8<INV>(v);
    else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 2) dft2<INV>(v[0], v[1]);
}

// v[k] *= W_B^{n2 k} (conjugated when CONJ) for k = 1..R-1, n2 < B / R.  tw[h + p] holds
// exp(-2 pi i p / (2h)) for p < h; the products n2 k read from the table stay below B / 2,
// the others are formed as w^{4a + b} = w^{4a} w^b.
template <int R, int B, bool CONJ, class E>
__device__ __forceinline__ void twiddle(E (&v)[R], const float2 *__restrict__ tw, int n2)
{
    const float2 *t = tw + (B >> 1);
    auto ld = [&](int j) {
        float2 w = __ldg(&t[j]);
        if (CONJ) w.y = -w.y;
        return w;
    };
    if constexpr (R == 2) {
        v[1] = e_mul(v[1], ld(n2));
    } else if constexpr (R == 4) {
        const float2 w1 = ld(n2), w2 = ld(2 * n2);
        v[1] = e_mul(v[1], w1);
        v[2] = e_mul(v[2], w2);
        v[3] = e_mul(v[3], cmulf(w1, w2));
    } else {
        const float2 w1 = ld(n2), w2 = ld(2 * n2), w3 = ld(3 * n2), w4 = ld(4 * n2);
        v[1] = e_mul(v[1], w1);
        v[2] = e_mul(v[2], w2);
        v[3] = e_mul(v[3], w3);
        float2 wa = w4;
#pragma unroll
        for (int a = 4; a < R; a += 4) {
            if (a > 4) wa = cmulf(wa, w4);
            v[a] = e_mul(v[a], wa);
            v[a + 1] = e_mul(v[a + 1], cmulf(wa, w1));
            v[a + 2] = e_mul(v[a + 2], cmulf(wa, w2));
            v[a + 3] = e_mul(v[a + 3], cmulf(wa, w3));
        }
    }
}

// Shared-memory element access of a 2^L buffer.
template <int L, class E = float2>
struct Smem {
    E *x;
    __device__ __forceinline__ E operator()(int p) const { return x[Geo<L>::sp(p)]; }
    __device__ __forceinline__ void operator()(int p, E v) const { x[Geo<L>::sp(p)] = v; }
};

template <class T> struct is_smem { static constexpr bool value = false; };
template <int L, class E> struct is_smem<Smem<L, E>> { static constexpr bool value = true; };

// sp(base + r S) = sp(base) + r * stride for S >= 16 (S a multiple of 16; the top digit is
// either constant over the block or equal to r when S is the top stride M / 16)
template <int L, int S>
__host__ __device__ constexpr int smem_stride() { return S + S / 16 + ((L >= 8 && S == (1 << L) / 16) ? 1 : 0); }

// DIF pass I (ADJ false: R-point DFT, then twiddles) or the adjoint of it (ADJ true:
// conjugate twiddles, then the inverse-sign R-point DFT).  Elements are read through ld(p)
// and written through st(p, v): shared memory, or the first/last pass fused with global
// input/output.  The last pass of a radix below 16 (stride 1) gives each thread 16 consecutive
// elements, 16 / R groups.
template <class E, int L, int I, bool ADJ, class Ld, class St>
__device__ __forceinline__ void pass(const float2 *__restrict__ tw, Ld ld, St st)
{
    using G = Geo<L>;
    constexpr int R = 1 << G::rb(I), S = G::S(I), B = R * S;
    if constexpr (S == 1 && R < 16 && G::M >= 16) {
        constexpr int units = G::M / 16;
        for (int u = threadIdx.x; u < units; u += blockDim.x) {
            E v[16];
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = ld(16 * u + r);
#pragma unroll
            for (int q = 0; q < 16 / R; ++q) {
                E w[R];
#pragma unroll
                for (int r = 0; r < R; ++r) w[r] = v[q * R + r];
                dft<R, ADJ>(w);
#pragma unroll
                for (int r = 0; r < R; ++r) v[q * R + r] = w[r];
            }
#pragma unroll
            for (int r = 0; r < 16; ++r) st(16 * u + r, v[r]);
        }
    } else {
        constexpr int groups = G::M / R;
        for (int g = threadIdx.x; g < groups; g += blockDim.x) {
            const int n2 = g & (S - 1);
            const int base = (g - n2) * R + n2;
            E v[R];
            if constexpr (is_smem<Ld>::value && S >= 16) {
                const E *p0 = ld.x + G::sp(base);
#pragma unroll
                for (int r = 0; r < R; ++r) v[r] = p0[r * smem_stride<L, S>()];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) v[r] = ld(base + r * S);
            }
            if constexpr (!ADJ) {
                dft<R, false>(v);
                if constexpr (S > 1) twiddle<R, B, false>(v, tw, n2);
            } else {
                if constexpr (S > 1) twiddle<R, B, true>(v, tw, n2);
                dft<R, true>(v);
            }
            if constexpr (is_smem<St>::value && S >= 16) {
                E *p0 = st.x + G::sp(base);
#pragma unroll
                for (int r = 0; r < R; ++r) p0[r * smem_stride<L, S>()] = v[r];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) st(base + r * S, v[r]);
            }
        }
    }
    __syncthreads();
}

// Forward DIF passes I..I1-1; pass I reads through ld, the others from shared memory.
template <int L, int I, int I1, class E, class Ld>
__device__ __forceinline__ void dif_passes(E *x, const float2 *__restrict__ tw, Ld ld)
{
    if constexpr (I < I1) {
        pass<E, L, I, false>(tw, ld, Smem<L, E>{x});
        dif_passes<L, I + 1, I1>(x, tw, Smem<L, E>{x});
    }
}

// Adjoint passes for DIF passes I down to 0; the last of them (pass 0) writes through st.
template <int L, int I, class E, class St>
__device__ __forceinline__ void adj_passes(E *x, const float2 *__restrict__ tw, St st)
{
    if constexpr (I == 0) {
        pass<E, L, 0, true>(tw, Smem<L, E>{x}, st);
    } else if constexpr (I > 0) {
        pass<E, L, I, true>(tw, Smem<L, E>{x}, Smem<L, E>{x});
        adj_passes<L, I - 1>(x, tw, st);
    }
}

// Forward DIF: natural-order input read through ld(k) by the first pass, digit-reversed
// spectrum out in x.
template <int L, class E, class Ld>
__device__ __forceinline__ void dif(E *x, const float2 *__restrict__ tw, Ld ld)
{
    dif_passes<L, 0, Geo<L>::NP>(x, tw, ld);
}

// Adjoint of dif: digit-reversed spectrum in x, M x inverse DFT out in natural order,
// written through st(k, v) by the last pass.
template <int L, class E, class St>
__device__ __forceinline__ void adj(E *x, const float2 *__restrict__ tw, St st)
{
    adj_passes<L, Geo<L>::NP - 1>(x, tw, st);
}

// The last DIF pass, the pointwise product with the spectrum fb (digit-reversed positions,
// conjugated when CONJ) and the first adjoint pass, fused: blocks of R points, no twiddles;
// a thread takes 16 consecutive points (16 / R blocks).  Elements are read through ld and
// written through st (shared memory unless the transform has this single pass).
template <int L, bool CONJ, class E, class Ld, class St>
__device__ __forceinline__ void middle(const float2 *__restrict__ fb, Ld ld, St st)
{
    constexpr int R = 1 << Geo<L>::LAST, P = Geo<L>::M >= 16 ? 16 : Geo<L>::M, units = Geo<L>::M / P;
    for (int u = threadIdx.x; u < units; u += blockDim.x) {
        E v[P];
#pragma unroll
        for (int r = 0; r < P; ++r) v[r] = ld(P * u + r);
        // the unit's P spectrum values (16-byte loads when they are 16 consecutive entries)
        float2 fv[P];
        if constexpr (P == 16) {
            const float4 *f4 = reinterpret_cast<const float4 *>(fb + P * u);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const float4 t = __ldg(&f4[r]);
                fv[2 * r] = make_float2(t.x, t.y);
                fv[2 * r + 1] = make_float2(t.z, t.w);
            }
        } else {
#pragma unroll
            for (int r = 0; r < P; ++r) fv[r] = __ldg(&fb[P * u + r]);
        }
#pragma unroll
        for (int q = 0; q < P / R; ++q) {
            E w[R];
#pragma unroll
            for (int r = 0; r < R; ++r) w[r] = v[q * R + r];
            dft<R, false>(w);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float2 f = fv[q * R + r];
                if (CONJ) f.y = -f.y;
                w[r] = e_mul(w[r], f);
            }
            dft<R, true>(w);
#pragma unroll
            for (int r = 0; r < R; ++r) v[q * R + r] = w[r];
        }
#pragma unroll
        for (int r = 0; r < P; ++r) st(P * u + r, v[r]);
    }
    __syncthreads();
}

// The value of the neighbour lane (lane ^ 1) of the same warp.
__device__ __forceinline__ float2 shfl_x1(float2 a)
{
    return make_float2(__shfl_xor_sync(0xffffffffu, a.x, 1), __shfl_xor_sync(0xffffffffu, a.y, 1));
}
__device__ __forceinline__ cpair shfl_x1(cpair a) { return cpair{shfl_x1(a.re), shfl_x1(a.im)}; }

// Trade halves with the neighbour lane: the even lane sends v[8 + k] and receives the odd
// lane's v[k] in its place; the odd lane sends v[k] and receives the even lane's v[8 + k] in
// its place (k < 8).  Applied twice it restores both lanes.
template <class E>
__device__ __forceinline__ void trade_halves(E (&v)[16], bool odd)
{
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const E r = shfl_x1(odd ? v[k] : v[8 + k]);
        if (odd) v[k] = r;
        else v[8 + k] = r;
    }
}

// For L = 4 K + 1 >= 9, whose last DIF pass is a radix-2 step: DIF pass NP - 2 (radix 16,
// stride 2), the radix-2 step, the pointwise product with fb, and the adjoints of the radix-2
// step and of pass NP - 2, all in registers -- the same operations in the same order as
// pass + middle + adjoint pass, without the two shared-memory round trips between them.
// Groups g = 2t and 2t + 1 of pass NP - 2 (neighbour lanes of one warp: the group count is a
// multiple of 32) hold positions 32t + 2r and 32t + 2r + 1 (r < 16), i.e. the two halves of
// the 16 radix-2 blocks (32t + 2r, 32t + 2r + 1); the even lane takes blocks r < 8 and the
// odd lane blocks r >= 8 (positions 16g + 2k, 16g + 2k + 1, k < 8, in both cases), trading
// halves with the neighbour lane before and after.  Reads through ld and writes through st
// (shared memory).
template <int L, bool CONJ, class E, class Ld, class St>
__device__ __forceinline__ void middle_r2(const float2 *__restrict__ tw, const float2 *__restrict__ fb, Ld ld, St st)
{
    using G = Geo<L>;
    constexpr int I = G::NP - 2, R = 16, S = G::S(I), B = R * S, groups = G::M / R;
    static_assert(G::LAST == 1 && S == 2 && groups % 32 == 0, "fused radix-2 middle needs L = 4K + 1 >= 9");
    for (int g = threadIdx.x; g < groups; g += blockDim.x) {  // warp-uniform trip count
        const int n2 = g & 1;
        const bool odd = n2 != 0;
        const int base = (g - n2) * R + n2;
        E v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = ld(base + r * S);
        dft<R, false>(v);
        twiddle<R, B, false>(v, tw, n2);
        trade_halves(v, odd);
        // block k of this lane is (v[k], v[8 + k]); its spectrum values are fb[16 g + 2k + {0, 1}]
        const float4 *f4 = reinterpret_cast<const float4 *>(fb + 16 * g);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float4 t = __ldg(&f4[k]);
            float2 f0 = make_float2(t.x, t.y), f1 = make_float2(t.z, t.w);
            if (CONJ) {
                f0.y = -f0.y;
                f1.y = -f1.y;
            }
            E a = v[k], b = v[8 + k];
            dft2<false>(a, b);
            a = e_mul(a, f0);
            b = e_mul(b, f1);
            dft2<true>(a, b);
            v[k] = a;
            v[8 + k] = b;
        }
        trade_halves(v, odd);
        twiddle<R, B, true>(v, tw, n2);
        dft<R, true>(v);
#pragma unroll
        for (int r = 0; r < R; ++r) st(base + r * S, v[r]);
    }
    __syncthreads();
}

// M times the circular convolution of the input (natural order, read through ld) with the
// sequence whose DIF spectrum fb holds (digit-reversed positions; conjugated when CONJ).
// The result, in natural order, is written through st.
template <int L, bool CONJ, class E, class Ld, class St>
__device__ __forceinline__ void convolve(E *x, const float2 *__restrict__ tw, const float2 *__restrict__ fb, Ld ld,
                                         St st)
{
    constexpr int NP = Geo<L>::NP;
    if constexpr (NP == 1) {
        middle<L, CONJ, E>(fb, ld, st);
    } else if constexpr (Geo<L>::LAST == 1 && L >= 9) {
        // radix-16 passes down to stride 32, the fused stride-2 pass / radix-2 product step,
        // then the adjoint passes from stride 32 up
        dif_passes<L, 0, NP - 2>(x, tw, ld);
        middle_r2<L, CONJ, E>(tw, fb, Smem<L, E>{x}, Smem<L, E>{x});
        adj_passes<L, NP - 3>(x, tw, st);
    } else {
        dif_passes<L, 0, NP - 1>(x, tw, ld);
        middle<L, CONJ, E>(fb, Smem<L, E>{x}, Smem<L, E>{x});
        adj_passes<L, NP - 2>(x, tw, st);
    }
}

}  // namespace fft
}  // namespace arkcos
