// Batched mixed-length ring FFTs (Sec. 4.1: real-to-complex FFT of every ring, length 4i in
// the polar caps and 4 nside on the equatorial belt; the inverse after the ring-band sum).
//
// One CTA owns one ring pair (j, R-1-j): mirror rings have the same length and offset, so
// their two real rings are packed as the real and imaginary parts of one complex sequence
// and split afterwards by Hermitian symmetry.  The CTA loops over all maps of the batch.
// Transforms run in shared memory over a power-of-two buffer M:
//   - power-of-two rings (M = n): one decimation-in-frequency (DIF) transform (forward) or one
//     decimation-in-time (DIT) transform from bit-reversed input (inverse);
//   - other lengths: Bluestein's chirp-z algorithm (1970) with M >= 2n - 1: DIF of the
//     chirped sequence (bit-reversed spectrum), pointwise product with the chirp spectrum held
//     in registers (same bit-reversed positions, computed once per CTA), DIT back to natural
//     order -- no explicit bit-reversal pass.
// Each pass fuses three radix-2 stages on eight elements in registers (radix 2^3).  Shared
// memory positions are XOR-swizzled within aligned groups of 16 complex values so that the
// natural, bit-reversed and every radix-8 stride pattern of a warp is free of bank conflicts.
// The chirps and first-pixel phases of a ring are tabulated once per CTA in shared memory
// and reused by every map of the batch.
// Epilogues fold in the first-pixel phase exp(-i m phi0) (Eq. fftrot), the ring weight and,
// on the inverse side, the Sec. 4.3 fold of super-Nyquist modes.
#include "device_common.cuh"

namespace arkcos {

namespace {

constexpr int kFbPer = 16;  // chirp-spectrum elements per thread (M <= 16 * blockDim)

__device__ __forceinline__ int brev(int e, int logM)
{
    return (int)(__brev((unsigned)e) >> (32 - logM));
}

// Shared-memory position of element i of a 2^L buffer: bits 0..3 XORed with bits 3..6 and with
// the top four bits (a bijection for L >= 8; identity for smaller buffers).
__device__ __forceinline__ int swz(int i, int L)
{
    return L >= 8 ? i ^ (((i >> 3) ^ (i >> (L - 4))) & 15) : i;
}

__device__ __forceinline__ float2 twid(const float2 *__restrict__ tw, int half, int p, bool inv)
{
    float2 w = __ldg(&tw[half + p]);  // exp(-2 pi i p / (2 half))
    if (inv) w.y = -w.y;
    return w;
}

// DIF butterfly: (u, v) -> (u + v, (u - v) w)
__device__ __forceinline__ void bf_dif(float2 &u, float2 &v, float2 w)
{
    const float2 s = caddf(u, v), d = csubf(u, v);
    u = s;
    v = cmulf(d, w);
}
// DIT butterfly: (u, v) -> (u + w v, u - w v)
__device__ __forceinline__ void bf_dit(float2 &u, float2 &v, float2 w)
{
    const float2 t = cmulf(v, w);
    v = csubf(u, t);
    u = caddf(u, t);
}

// Multiplication by the constant eighth roots of unity W_8^r = exp(-2 pi i r / 8) (inv: conj).
template <int R, bool INV>
__device__ __forceinline__ float2 rot8(float2 a)
{
    constexpr float h = 0.70710678118654752f;
    if (R == 0) return a;
    if (R == 2) return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);  // * (+-i)
    if (R == 1)
        return INV ? make_float2(h * (a.x - a.y), h * (a.x + a.y))
                   : make_float2(h * (a.x + a.y), h * (a.y - a.x));
    // R == 3: W_8^3 = (-1 - i)/sqrt2, conj = (-1 + i)/sqrt2
    return INV ? make_float2(-h * (a.x + a.y), h * (a.x - a.y))
               : make_float2(h * (a.y - a.x), -h * (a.x + a.y));
}

__device__ __forceinline__ float2 csq(float2 a) { return make_float2(a.x * a.x - a.y * a.y, 2.f * a.x * a.y); }

// One radix-2^3 DIF group: stages of half size 4q, 2q, q on v[0..7] = x[i0 + r q].  The
// stage twiddles are W_{8q}^{pos + r q} = w W_8^r, W_{4q}^{pos + r q} = w^2 W_4^r and
// W_{2q}^{pos} = w^4 with w = W_{8q}^{pos}: one table load per group.
template <bool INV>
__device__ __forceinline__ void dif8(float2 (&v)[8], float2 w)
{
    const float2 w2 = csq(w), w4 = csq(w2);
    float2 d;
    // stage 1 (half 4q)
    d = csubf(v[0], v[4]); v[0] = caddf(v[0], v[4]); v[4] = cmulf(d, w);
    d = csubf(v[1], v[5]); v[1] = caddf(v[1], v[5]); v[5] = cmulf(rot8<1, INV>(d), w);
    d = csubf(v[2], v[6]); v[2] = caddf(v[2], v[6]); v[6] = cmulf(rot8<2, INV>(d), w);
    d = csubf(v[3], v[7]); v[3] = caddf(v[3], v[7]); v[7] = cmulf(rot8<3, INV>(d), w);
    // stage 2 (half 2q): twiddles w2 (r even) and w2 W_4 (r odd)
    d = csubf(v[0], v[2]); v[0] = caddf(v[0], v[2]); v[2] = cmulf(d, w2);
    d = csubf(v[1], v[3]); v[1] = caddf(v[1], v[3]); v[3] = cmulf(rot8<2, INV>(d), w2);
    d = csubf(v[4], v[6]); v[4] = caddf(v[4], v[6]); v[6] = cmulf(d, w2);
    d = csubf(v[5], v[7]); v[5] = caddf(v[5], v[7]); v[7] = cmulf(rot8<2, INV>(d), w2);
    // stage 3 (half q)
#pragma unroll
    for (int r = 0; r < 8; r += 2) {
        d = csubf(v[r], v[r + 1]);
        v[r] = caddf(v[r], v[r + 1]);
        v[r + 1] = cmulf(d, w4);
    }
}

// One radix-2^3 DIT group: stages of half size q, 2q, 4q (the transpose of dif8).
template <bool INV>
__device__ __forceinline__ void dit8(float2 (&v)[8], float2 w)
{
    const float2 w2 = csq(w), w4 = csq(w2);
    float2 t;
#pragma unroll
    for (int r = 0; r < 8; r += 2) {
        t = cmulf(v[r + 1], w4);
        v[r + 1] = csubf(v[r], t);
        v[r] = caddf(v[r], t);
    }
    t = cmulf(v[2], w2); v[2] = csubf(v[0], t); v[0] = caddf(v[0], t);
    t = rot8<2, INV>(cmulf(v[3], w2)); v[3] = csubf(v[1], t); v[1] = caddf(v[1], t);
    t = cmulf(v[6], w2); v[6] = csubf(v[4], t); v[4] = caddf(v[4], t);
    t = rot8<2, INV>(cmulf(v[7], w2)); v[7] = csubf(v[5], t); v[5] = caddf(v[5], t);
    t = cmulf(v[4], w); v[4] = csubf(v[0], t); v[0] = caddf(v[0], t);
    t = rot8<1, INV>(cmulf(v[5], w)); v[5] = csubf(v[1], t); v[1] = caddf(v[1], t);
    t = rot8<2, INV>(cmulf(v[6], w)); v[6] = csubf(v[2], t); v[2] = caddf(v[2], t);
    t = rot8<3, INV>(cmulf(v[7], w)); v[7] = csubf(v[3], t); v[3] = caddf(v[3], t);
}

// In-place DIF over M = 2^logM: natural-order input, bit-reversed output.  Stages with half
// sizes M/2, M/4, ..., 1, fused three (or fewer, for the last pass) at a time.
template <bool INV>
__device__ void fft_dif(float2 *x, int M, int logM, const float2 *__restrict__ tw)
{
    int left = logM;
    int h = M >> 1;  // half size of the first stage of the pass
    while (left > 0) {
        const int ns = left >= 3 ? 3 : left;
        const int q = h >> (ns - 1);  // half size of the last stage of the pass
        const int groups = M >> ns;
        for (int g = threadIdx.x; g < groups; g += blockDim.x) {
            const int pos = g & (q - 1);
            const int i0 = ((g - pos) << ns) | pos;
            float2 v[8];
            if (ns == 3) {
#pragma unroll
                for (int r = 0; r < 8; ++r) v[r] = x[swz(i0 + r * q, logM)];
                dif8<INV>(v, twid(tw, 4 * q, pos, INV));
#pragma unroll
                for (int r = 0; r < 8; ++r) x[swz(i0 + r * q, logM)] = v[r];
            } else if (ns == 2) {
#pragma unroll
                for (int r = 0; r < 4; ++r) v[r] = x[swz(i0 + r * q, logM)];
#pragma unroll
                for (int r = 0; r < 2; ++r) bf_dif(v[r], v[r + 2], twid(tw, 2 * q, pos + r * q, INV));
                const float2 w = twid(tw, q, pos, INV);
                bf_dif(v[0], v[1], w);
                bf_dif(v[2], v[3], w);
#pragma unroll
                for (int r = 0; r < 4; ++r) x[swz(i0 + r * q, logM)] = v[r];
            } else {
                v[0] = x[swz(i0, logM)];
                v[1] = x[swz(i0 + q, logM)];
                bf_dif(v[0], v[1], twid(tw, q, pos, INV));
                x[swz(i0, logM)] = v[0];
                x[swz(i0 + q, logM)] = v[1];
            }
        }
        __syncthreads();
        left -= ns;
        h = q >> 1;
    }
}

// In-place DIT over M = 2^logM: bit-reversed input, natural-order output.  Stages with half
// sizes 1, 2, ..., M/2, fused three (or fewer, for the last pass) at a time.
template <bool INV>
__device__ void fft_dit(float2 *x, int M, int logM, const float2 *__restrict__ tw)
{
    int left = logM;
    int q = 1;  // half size of the first stage of the pass
    while (left > 0) {
        const int ns = left >= 3 ? 3 : left;
        const int groups = M >> ns;
        for (int g = threadIdx.x; g < groups; g += blockDim.x) {
            const int pos = g & (q - 1);
            const int i0 = ((g - pos) << ns) | pos;
            float2 v[8];
            if (ns == 3) {
#pragma unroll
                for (int r = 0; r < 8; ++r) v[r] = x[swz(i0 + r * q, logM)];
                dit8<INV>(v, twid(tw, 4 * q, pos, INV));
#pragma unroll
                for (int r = 0; r < 8; ++r) x[swz(i0 + r * q, logM)] = v[r];
            } else if (ns == 2) {
#pragma unroll
                for (int r = 0; r < 4; ++r) v[r] = x[swz(i0 + r * q, logM)];
                const float2 w = twid(tw, q, pos, INV);
                bf_dit(v[0], v[1], w);
                bf_dit(v[2], v[3], w);
#pragma unroll
                for (int r = 0; r < 2; ++r) bf_dit(v[r], v[r + 2], twid(tw, 2 * q, pos + r * q, INV));
#pragma unroll
                for (int r = 0; r < 4; ++r) x[swz(i0 + r * q, logM)] = v[r];
            } else {
                v[0] = x[swz(i0, logM)];
                v[1] = x[swz(i0 + q, logM)];
                bf_dit(v[0], v[1], twid(tw, q, pos, INV));
                x[swz(i0, logM)] = v[0];
                x[swz(i0 + q, logM)] = v[1];
            }
        }
        __syncthreads();
        left -= ns;
        q <<= ns;
    }
}

// Spectrum of the Bluestein chirp b_k = conj(chirp[|k|]), |k| < n, circular in M, in
// bit-reversed order (DIF); element e = tid + r * blockDim lands in fb[r].
__device__ void chirp_spectrum(float2 *buf, int M, int logM, int n, const float2 *chirp,
                               const float2 *__restrict__ tw, float2 (&fb)[kFbPer])
{
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
        int kk = -1;
        if (k < n) kk = k;
        else if (k > M - n) kk = M - k;
        buf[swz(k, logM)] = kk < 0 ? make_float2(0.f, 0.f) : cconjf(chirp[kk]);
    }
    __syncthreads();
    fft_dif<false>(buf, M, logM, tw);
#pragma unroll
    for (int r = 0; r < kFbPer; ++r) {
        const int e = threadIdx.x + r * blockDim.x;
        fb[r] = e < M ? buf[swz(e, logM)] : make_float2(0.f, 0.f);
    }
    __syncthreads();
}

// Per-CTA tables of a ring of n pixels: chirp[k] = exp(sgn i pi k^2 / n) for k < n (Bluestein
// rings) and phase[m] = exp(sgn i pi m / n) for m <= n/2 (rings with a half-pixel offset).
__device__ void ring_tables(float2 *chirp, float2 *phase, int n, bool blu, bool hs, int sgn)
{
    if (blu)
        for (int k = threadIdx.x; k < n; k += blockDim.x) chirp[k] = expipi_ratio(sgn * k * k, n);
    if (hs)
        for (int m = threadIdx.x; m <= n / 2; m += blockDim.x) phase[m] = expipi_ratio(sgn * m, n);
    __syncthreads();
}

// Bluestein convolution: buf holds the chirped sequence (natural order).  Afterwards
// buf[swz(m, logM)] = M * sum_q a_q b_{m-q} in natural order.
__device__ void bluestein_convolve(float2 *buf, int M, int logM, const float2 *__restrict__ tw,
                                   const float2 (&fb)[kFbPer])
{
    fft_dif<false>(buf, M, logM, tw);
#pragma unroll
    for (int r = 0; r < kFbPer; ++r) {
        const int e = threadIdx.x + r * blockDim.x;
        if (e < M) buf[swz(e, logM)] = cmulf(buf[swz(e, logM)], fb[r]);
    }
    __syncthreads();
    fft_dit<true>(buf, M, logM, tw);
}

// Buffer size of a ring: n itself when it is a power of two, else the Bluestein size.
__device__ __forceinline__ int ring_log2_buffer(int n)
{
    int l = 1;
    while ((1 << l) < n) ++l;
    if ((1 << l) == n) return l;
    l = 1;
    while ((1 << l) < 2 * n - 1) ++l;
    return l;
}

__global__ void __launch_bounds__(1024) k_fft_fwd(FftFwdArgs a)
{
    extern __shared__ float2 buf[];  // [a.M] transform buffer, then the ring's tables
    const int j = a.reps[blockIdx.x];
    const int j2 = a.R - 1 - j;
    const bool pair = j2 != j;
    const int n = a.rd.n[j];
    const int logM = ring_log2_buffer(n);  // a launch may cover several buffer sizes <= a.M
    const int M = 1 << logM;
    const bool blu = (M != n);
    const int hs = a.rd.hs[j];
    float2 *chirp = buf + a.M;                      // exp(-i pi k^2 / n)
    float2 *phase = chirp + (blu ? n : 0);          // exp(-i pi m / n)
    ring_tables(chirp, phase, n, blu, hs, -1);
    float2 fb[kFbPer];
    if (blu) chirp_spectrum(buf, M, logM, n, chirp, a.tw, fb);
    const float wsc = a.weight ? a.rd.w[j] : 1.0f;
    const bool zero = a.zero_poles && j == 0;
    const float inv_m = 1.0f / (float)M;
    for (int b = 0; b < a.B; ++b) {
        const float *m1 = a.map + (int64_t)b * a.npix + a.rd.poff[j];
        const float *m2 = a.map + (int64_t)b * a.npix + a.rd.poff[j2];
        for (int k = threadIdx.x; k < M; k += blockDim.x) {
            float2 v = make_float2(0.f, 0.f);
            if (k < n && !zero) {
                v.x = __ldg(&m1[k]);
                v.y = pair ? __ldg(&m2[k]) : 0.f;
                if (blu) v = cmulf(v, chirp[k]);
            }
            buf[swz(k, logM)] = v;
        }
        __syncthreads();
        if (blu) bluestein_convolve(buf, M, logM, a.tw, fb);
        else fft_dif<false>(buf, M, logM, a.tw);
        if (a.ext4) {
            // every kernel-grid mode m <= N/2: the periodic extension a_{m + qn} =
            // exp(-i q n phi0) a_m (ENHANCED) or the Nyquist-halved truncation (BASIC)
            float4 *o4 = a.spec4 + ((int64_t)b * a.nrep + j) * a.NH;
            for (int m = threadIdx.x; m < a.NH; m += blockDim.x) {
                int q = (int)__fdividef((float)m, (float)n);
                int mm = m - q * n;
                if (mm < 0) {
                    --q;
                    mm += n;
                } else if (mm >= n) {
                    ++q;
                    mm -= n;
                }
                const bool up = 2 * mm > n;
                const int mb = up ? n - mm : mm;  // base mode in [0, n/2]
                const int mn = mb == 0 ? 0 : n - mb;
                float2 zm, zn;
                if (blu) {
                    zm = cscalef(cmulf(buf[swz(mb, logM)], chirp[mb]), inv_m);
                    zn = cscalef(cmulf(buf[swz(mn, logM)], chirp[mn]), inv_m);
                } else {
                    zm = buf[swz(brev(mb, logM), logM)];
                    zn = buf[swz(brev(mn, logM), logM)];
                }
                const float2 ph = hs ? phase[mb] : make_float2(1.f, 0.f);
                float2 ea = cmulf(make_float2(0.5f * (zm.x + zn.x), 0.5f * (zm.y - zn.y)), ph);
                // the middle ring is its own mirror: its row holds (a, a)
                float2 eb = pair ? cmulf(make_float2(0.5f * (zm.y + zn.y), -0.5f * (zm.x - zn.x)), ph)
                                 : ea;
                float sc = wsc;
                if (a.basic) {
                    if (q > 0 || up) sc = 0.f;
                    else if (2 * mm == n && n < a.N) sc *= 0.5f;
                } else {
                    if (up) {
                        ea.y = -ea.y;
                        eb.y = -eb.y;
                    }
                    if (hs && ((q + (up ? 1 : 0)) & 1)) sc = -sc;
                }
                o4[m] = make_float4(sc * ea.x, sc * ea.y, sc * eb.x, sc * eb.y);
            }
            __syncthreads();
            continue;
        }
        float2 *s1 = a.spec + (int64_t)b * a.nspec + a.rd.soff[j];
        float2 *s2 = a.spec + (int64_t)b * a.nspec + a.rd.soff[j2];
        for (int m = threadIdx.x; m <= n / 2; m += blockDim.x) {
            const int mn = m == 0 ? 0 : n - m;
            float2 zm, zn;
            if (blu) {
                zm = cscalef(cmulf(buf[swz(m, logM)], chirp[m]), inv_m);
                zn = cscalef(cmulf(buf[swz(mn, logM)], chirp[mn]), inv_m);
            } else {
                zm = buf[swz(brev(m, logM), logM)];
                zn = buf[swz(brev(mn, logM), logM)];
            }
            const float2 ph = hs ? phase[m] : make_float2(1.f, 0.f);
            const float2 ea = make_float2(0.5f * (zm.x + zn.x), 0.5f * (zm.y - zn.y));
            s1[m] = cscalef(cmulf(ea, ph), wsc);
            if (pair) {
                // (Z_m - conj Z_{n-m}) / (2i)
                const float2 eb = make_float2(0.5f * (zm.y + zn.y), -0.5f * (zm.x - zn.x));
                s2[m] = cscalef(cmulf(eb, ph), wsc);
            }
        }
        __syncthreads();
    }
}

// Folded output coefficient D_{mm}, mm in [0, n/2], of ring i: the modes m of the full
// kernel grid (|m| <= N/2) that alias to mm on a ring of n pixels, each taken after the
// reverse phase shift exp(+i m phi0_i) (Sec. 4.1) and summed (Sec. 4.3).  The BASIC
// variant keeps only |m| <= n/2 (Sec. 4.1, truncation at the ring's Nyquist frequency).
// c may live in global or shared memory.
__device__ __forceinline__ float2 folded_coeff(const float2 *c, int mm, int n, int hs, float2 ph,
                                               int N, bool basic)
{
    const int nyq = N / 2;
    // reverse phase exp(+i m pi / n) for the aliases m = mm + t n is (-1)^t ph, ph =
    // exp(i pi mm / n) (1 without offset), and for m = t n - mm it is (-1)^t conj(ph)
    if (basic) {
        float2 d = c[mm];
        if (mm == 0) d.y = 0.f;  // the m = 0 term of a real ring
        d = cmulf(d, ph);
        if (2 * mm == n) d.y = 0.f;  // (d + conj d) / 2
        return d;
    }
    float2 acc = make_float2(0.f, 0.f);
    float sg = 1.f;
    for (int m = mm; m <= nyq; m += n) {
        float2 d = c[m];
        if (m == 0) d.y = 0.f;  // the m = 0 term of a real ring
        const float h = ((m == nyq) ? 0.5f : 1.0f) * sg;
        acc.x += h * d.x;
        acc.y += h * d.y;
        if (hs) sg = -sg;
    }
    acc = cmulf(acc, ph);
    // negative modes -m, m = t n - mm (t >= 1): conj(c_m exp(i m pi/n)) = (-1)^t conj(c_m) ph
    float2 neg = make_float2(0.f, 0.f);
    sg = hs ? -1.f : 1.f;
    for (int m = n - mm; m <= nyq; m += n) {
        const float2 d = c[m];
        const float h = ((m == nyq) ? 0.5f : 1.0f) * sg;
        neg.x += h * d.x;
        neg.y += h * d.y;
        if (hs) sg = -sg;
    }
    neg = cmulf(neg, cconjf(ph));  // conj(neg * conj(ph)) = conj(neg) * ph
    acc.x += neg.x;
    acc.y -= neg.y;
    return acc;
}

__global__ void __launch_bounds__(1024) k_fft_inv(FftInvArgs a)
{
    extern __shared__ float2 buf[];  // [a.M] buffer | [2 NH] staged coefficients | tables
    const int i = a.reps[blockIdx.x];
    if (a.skip_poles && i == 0) return;  // rings 0 and R-1 come from the pole kernel
    const int i2 = a.R - 1 - i;
    const bool pair = i2 != i;
    const int n = a.rd.n[i];
    const int logM = ring_log2_buffer(n);
    const int M = 1 << logM;
    const bool blu = (M != n);
    const int hs = a.rd.hs[i];
    // rings much shorter than the kernel grid fold many modes onto each frequency: stage the
    // coefficients in shared memory with coalesced loads first
    const bool stage = a.stage_c && !a.basic && 4 * n < a.N;
    float2 *cs1 = buf + a.M, *cs2 = cs1 + a.NH;
    float2 *chirp = buf + a.M + (a.stage_c ? 2 * a.NH : 0);  // exp(+i pi k^2 / n)
    float2 *phase = chirp + (blu ? n : 0);                    // exp(+i pi m / n)
    ring_tables(chirp, phase, n, blu, hs, +1);
    float2 fb[kFbPer];
    if (blu) chirp_spectrum(buf, M, logM, n, chirp, a.tw, fb);
    const float wsc = a.weight ? a.rd.w[i] : 1.0f;
    const float inv_m = 1.0f / (float)M;
    for (int b = 0; b < a.B; ++b) {
        const float2 *c1 = a.c + ((int64_t)b * a.R + i) * a.NH;
        const float2 *c2 = a.c + ((int64_t)b * a.R + i2) * a.NH;
        if (stage) {
            for (int m = threadIdx.x; m < a.NH; m += blockDim.x) {
                cs1[m] = __ldg(&c1[m]);
                cs2[m] = pair ? __ldg(&c2[m]) : make_float2(0.f, 0.f);
            }
            __syncthreads();
            c1 = cs1;
            c2 = cs2;
        }
        for (int k = threadIdx.x; k < M; k += blockDim.x) {
            float2 v = make_float2(0.f, 0.f);
            if (k < n) {
                const bool up = 2 * k > n;
                const int mm = up ? n - k : k;
                const float2 ph = hs ? phase[mm] : make_float2(1.f, 0.f);
                float2 d1 = folded_coeff(c1, mm, n, hs, ph, a.N, a.basic);
                float2 d2 = pair ? folded_coeff(c2, mm, n, hs, ph, a.N, a.basic) : make_float2(0.f, 0.f);
                if (up) {
                    d1.y = -d1.y;
                    d2.y = -d2.y;
                }
                // X = D(i) + i D(i2)
                v = make_float2(wsc * (d1.x - d2.y), wsc * (d1.y + d2.x));
                if (blu) v = cmulf(v, chirp[k]);
            }
            // DIT wants bit-reversed input (power-of-two rings); Bluestein takes natural order
            buf[swz(blu ? k : brev(k, logM), logM)] = v;
        }
        __syncthreads();
        if (blu) bluestein_convolve(buf, M, logM, a.tw, fb);
        else fft_dit<true>(buf, M, logM, a.tw);
        float *o1 = a.map + (int64_t)b * a.npix + a.rd.poff[i];
        float *o2 = a.map + (int64_t)b * a.npix + a.rd.poff[i2];
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            float2 z = buf[swz(p, logM)];
            if (blu) z = cscalef(cmulf(z, chirp[p]), inv_m);
            o1[p] = z.x;
            if (pair) o2[p] = z.y;
        }
        __syncthreads();
    }
}

}  // namespace

size_t fft_smem_bytes(int M, int N, bool stage_c, int tab)
{
    size_t words = (size_t)M + (size_t)tab;
    if (stage_c) words += 2 * (size_t)(N / 2 + 1);
    return words * sizeof(float2);
}

static cudaError_t set_smem(const void *fn, size_t bytes)
{
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_fft_fwd(const FftFwdArgs &a, int count, int threads, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const size_t smem = fft_smem_bytes(a.M, a.N, false, a.tab);
    cudaError_t e = set_smem((const void *)k_fft_fwd, smem);
    if (e != cudaSuccess) return e;
    k_fft_fwd<<<count, threads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fft_inv(const FftInvArgs &a, int count, int threads, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const size_t smem = fft_smem_bytes(a.M, a.N, a.stage_c != 0, a.tab);
    cudaError_t e = set_smem((const void *)k_fft_inv, smem);
    if (e != cudaSuccess) return e;
    k_fft_inv<<<count, threads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace arkcos
