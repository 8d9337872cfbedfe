// Inverse ring transforms after the ring-band sum (Sec. 4.1), with the Sec. 4.3 fold of the
// kernel-grid modes onto each ring's own frequencies.
#include "ring_common.cuh"

namespace arkcos {

namespace {

using fft::cpair;
using ring::chirp_at;

// Folded output coefficient D_{mm}, mm in [0, n/2], of ring i: the modes m of the full
// kernel grid (|m| <= N/2) that alias to mm on a ring of n pixels, each taken after the
// reverse phase shift exp(+i m phi0_i) (Sec. 4.1) and summed (Sec. 4.3).  The BASIC
// variant keeps only |m| <= n/2 (Sec. 4.1, truncation at the ring's Nyquist frequency).
// c may live in global or shared memory; ph = exp(i pi mm / n) for half-pixel rings, else 1.
__device__ __forceinline__ float2 folded_coeff(const float2 *c, int mm, int n, int hs, float2 ph, int N, bool basic)
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

// The same fold for every mm of a short ring pair with the whole CTA, straight from the
// coefficients in global memory: thread w = ch nh + mm sums the aliases t = ch, ch + C, ... of
// bin mm for both rings (consecutive threads read consecutive modes), then each bin adds its
// C partial sums (part: 2 C (n/2 + 1) <= 2 blockDim entries) in chunk order.  c1, c2 are the
// coefficients of rings i and i2 (c2 unused without a pair); ph(mm) the reverse phase of bin mm.
template <class Ph>
__device__ __forceinline__ void fold_all(const float2 *__restrict__ c1, const float2 *__restrict__ c2, bool pair,
                                         int n, int hs, int N, Ph ph, float2 *D1, float2 *D2, float4 *part)
{
    const int nh = n / 2 + 1, nyq = N / 2, T = blockDim.x;
    int C = 1;
    while (2 * C * nh <= T) C *= 2;
    for (int w = threadIdx.x; w < nh * C; w += T) {
        const int ch = w / nh, mm = w - ch * nh;
        float2 p1 = make_float2(0.f, 0.f), p2 = p1, q1 = p1, q2 = p1;
        // positive aliases m = mm + t n: weight (-1)^t with the offset, 1/2 at the Nyquist mode,
        // and negative aliases -m, m = t n - mm (t >= 1); four aliases of each kind loaded
        // together
        constexpr int U = 4;
        for (int t0 = ch;; t0 += U * C) {
            if (mm + t0 * n > nyq && (t0 + 1) * n - mm > nyq) break;
            float2 d1[U], d2[U], e1[U], e2[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int t = t0 + u * C, m = mm + t * n, mn = (t + 1) * n - mm;
                d1[u] = m <= nyq ? __ldg(&c1[m]) : make_float2(0.f, 0.f);
                d2[u] = pair && m <= nyq ? __ldg(&c2[m]) : make_float2(0.f, 0.f);
                e1[u] = mn <= nyq ? __ldg(&c1[mn]) : make_float2(0.f, 0.f);
                e2[u] = pair && mn <= nyq ? __ldg(&c2[mn]) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int t = t0 + u * C, m = mm + t * n, mn = (t + 1) * n - mm;
                const float sg = (hs && (t & 1)) ? -1.f : 1.f;
                const float h = (m == nyq ? 0.5f : 1.0f) * sg;
                if (m == 0) d1[u].y = d2[u].y = 0.f;  // the m = 0 term of a real ring
                p1.x += h * d1[u].x;
                p1.y += h * d1[u].y;
                p2.x += h * d2[u].x;
                p2.y += h * d2[u].y;
                const float hq = (mn == nyq ? 0.5f : 1.0f) * (hs ? -sg : 1.f);  // (-1)^(t+1)
                q1.x += hq * e1[u].x;
                q1.y += hq * e1[u].y;
                q2.x += hq * e2[u].x;
                q2.y += hq * e2[u].y;
            }
        }
        if (C == 1) {  // one thread per bin: finish it here
            const float2 pm = ph(mm);
            const float2 a1 = cmulf(p1, pm), g1 = cmulf(q1, cconjf(pm));
            const float2 a2 = cmulf(p2, pm), g2 = cmulf(q2, cconjf(pm));
            D1[mm] = make_float2(a1.x + g1.x, a1.y - g1.y);
            D2[mm] = pair ? make_float2(a2.x + g2.x, a2.y - g2.y) : make_float2(0.f, 0.f);
        } else {       // nh C <= blockDim partial sums
            part[2 * (mm * C + ch)] = make_float4(p1.x, p1.y, q1.x, q1.y);
            part[2 * (mm * C + ch) + 1] = make_float4(p2.x, p2.y, q2.x, q2.y);
        }
    }
    __syncthreads();
    if (C == 1) return;
    for (int mm = threadIdx.x; mm < nh; mm += T) {
        float4 s1 = make_float4(0.f, 0.f, 0.f, 0.f), s2 = s1;
        for (int ch = 0; ch < C; ++ch) {
            const float4 u = part[2 * (mm * C + ch)], v = part[2 * (mm * C + ch) + 1];
            s1.x += u.x; s1.y += u.y; s1.z += u.z; s1.w += u.w;
            s2.x += v.x; s2.y += v.y; s2.z += v.z; s2.w += v.w;
        }
        const float2 pm = ph(mm);
        float2 a1 = cmulf(make_float2(s1.x, s1.y), pm), g1 = cmulf(make_float2(s1.z, s1.w), cconjf(pm));
        float2 a2 = cmulf(make_float2(s2.x, s2.y), pm), g2 = cmulf(make_float2(s2.z, s2.w), cconjf(pm));
        D1[mm] = make_float2(a1.x + g1.x, a1.y - g1.y);
        D2[mm] = pair ? make_float2(a2.x + g2.x, a2.y - g2.y) : make_float2(0.f, 0.f);
    }
    __syncthreads();
}

// One output ring pair through the h-point inverse transforms of its two rings (lanes of a
// cpair): the folded half spectra X_k of both rings give
//   Z_k = E + i O,  E = X_k + conj X_{h-k},  O = (X_k - conj X_{h-k}) exp(2 pi i k / n),
// whose h-point inverse DFT (unnormalised) is z_q = x_2q + i x_2q+1.
struct InvCta {
    const FftInvArgs &a;
    cpair *buf;
    float2 *D1, *D2;
    float4 *part;
    const float2 *chirp, *phase, *fb;  // chirp of h (Bluestein rings), exp(+i pi m / n) for m <= n/2
    int i, i2, n, h, hs;
    bool pair, blu, stage;
    float wsc;

    // exp(+i pi m / n), 0 <= m <= n/2
    __device__ __forceinline__ float2 ph(int m) const { return phase[m]; }
    // the reverse phase of the first pixel (1 for rings without the half-pixel offset)
    __device__ __forceinline__ float2 rph(int m) const { return hs ? ph(m) : make_float2(1.f, 0.f); }

    template <int L>
    __device__ void run()
    {
        constexpr int M = 1 << L;
        const fft::Smem<L, cpair> sm{buf};
        const float inv_m = 1.0f / (float)M;
        const int bend = min(a.B, (int)(blockIdx.y + 1) * a.mchunk);
        const int nyq = a.N / 2;
        for (int b = blockIdx.y * a.mchunk; b < bend; ++b) {
            const float2 *c1 = a.c + ((int64_t)b * a.R + i) * a.NH;
            const float2 *c2 = a.c + ((int64_t)b * a.R + i2) * a.NH;
            if (b + 1 < bend) {
                // the next map's coefficient rows of both rings into L2 while this map is
                // transformed (128-byte lines)
                const char *p1 = reinterpret_cast<const char *>(c1 + (int64_t)a.R * a.NH);
                const char *p2 = reinterpret_cast<const char *>(c2 + (int64_t)a.R * a.NH);
                const int lines = (a.NH * 8 + 127) / 128;
                for (int l = threadIdx.x; l < 2 * lines; l += blockDim.x)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"((l < lines ? p1 : p2) + 128 * (l % lines)));
            }
            // short rings fold many modes onto each frequency: the whole CTA folds them first
            if (stage) fold_all(c1, c2, pair, n, hs, a.N, [&](int mm) { return rph(mm); }, D1, D2, part);
            // the folded coefficients D(mm) of ring and mirror, mm in [0, n/2], as lanes
            auto folded = [&](int mm) {
                float2 d1, d2;
                if (stage) {
                    d1 = D1[mm];
                    d2 = D2[mm];
                } else if (!a.basic && 2 * n > a.N) {
                    // rings longer than N/2 have at most one alias on each side (m = mm and
                    // m = n - mm): the fold of folded_coeff with its two terms written out
                    const int mn = n - mm;
                    const bool neg = mn <= nyq;
                    float2 x1 = __ldg(&c1[mm]), x2 = pair ? __ldg(&c2[mm]) : make_float2(0.f, 0.f);
                    const float2 y1 = neg ? __ldg(&c1[mn]) : make_float2(0.f, 0.f);
                    const float2 y2 = neg && pair ? __ldg(&c2[mn]) : make_float2(0.f, 0.f);
                    const float2 p = rph(mm);
                    const float hp = mm == nyq ? 0.5f : 1.0f;
                    const float hq = (mn == nyq ? 0.5f : 1.0f) * (hs ? -1.f : 1.f);
                    if (mm == 0) x1.y = x2.y = 0.f;  // the m = 0 term of a real ring
                    d1 = cmulf(cscalef(x1, hp), p);
                    d2 = cmulf(cscalef(x2, hp), p);
                    const float2 g1 = cmulf(cscalef(y1, hq), cconjf(p)), g2 = cmulf(cscalef(y2, hq), cconjf(p));
                    d1 = make_float2(d1.x + g1.x, d1.y - g1.y);
                    d2 = make_float2(d2.x + g2.x, d2.y - g2.y);
                } else {
                    const float2 p = rph(mm);
                    d1 = folded_coeff(c1, mm, n, hs, p, a.N, a.basic);
                    d2 = pair ? folded_coeff(c2, mm, n, hs, p, a.N, a.basic) : make_float2(0.f, 0.f);
                }
                return cpair{make_float2(d1.x, d2.x), make_float2(d1.y, d2.y)};
            };
            // transform input at k and h - k from the folded X_k and X_{h-k} of both rings
            auto emit = [&](auto put, int k, const cpair &xk, const cpair &xh) {
                using namespace fft;
                const float2 Er = caddf(xk.re, xh.re), Ei = csubf(xk.im, xh.im);
                const float2 Fr = csubf(xk.re, xh.re), Fi = caddf(xk.im, xh.im);
                const float2 v = ph(2 * k);  // exp(2 pi i k / n)
                const float2 Or = pfma(Fi, bcast(-v.y), pmul(Fr, bcast(v.x)));
                const float2 Oi = pfma(Fi, bcast(v.x), pmul(Fr, bcast(v.y)));
                const float2 ws = bcast(wsc);
                cpair zk{pmul(csubf(Er, Oi), ws), pmul(caddf(Ei, Or), ws)};
                if (blu) zk = e_mul(zk, chirp_at(chirp, k, h));
                put(k, zk);
                if (k > 0 && 2 * k < h) {
                    cpair zh{pmul(caddf(Er, Oi), ws), pmul(csubf(Or, Ei), ws)};
                    if (blu) zh = e_mul(zh, chirp_at(chirp, h - k, h));
                    put(h - k, zh);
                }
            };
            auto fill = [&](auto put) {
                constexpr int U = 4;  // values of k per thread whose loads are issued together
                if (!stage && n == a.N) {
                    // rings as long as the kernel grid: bin k < h takes the mode c_k alone (the
                    // BASIC truncation at the ring's Nyquist frequency and the ENHANCED fold
                    // coincide for these rings)
                    for (int k0 = threadIdx.x; 2 * k0 <= h; k0 += U * blockDim.x) {
                        float2 a1[U], a2[U], b1[U], b2[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int k = min(k0 + u * (int)blockDim.x, h / 2);
                            a1[u] = __ldg(&c1[k]);
                            b1[u] = __ldg(&c1[h - k]);
                            a2[u] = pair ? __ldg(&c2[k]) : make_float2(0.f, 0.f);
                            b2[u] = pair ? __ldg(&c2[h - k]) : make_float2(0.f, 0.f);
                        }
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int k = k0 + u * blockDim.x;
                            if (2 * k > h) break;
                            if (k == 0) continue;  // bins 0 and h (the Nyquist mode) below
                            const float2 p = rph(k), q = rph(h - k);
                            const float2 d1 = cmulf(a1[u], p), d2 = cmulf(a2[u], p);
                            const float2 e1 = cmulf(b1[u], q), e2 = cmulf(b2[u], q);
                            emit(put, k, cpair{make_float2(d1.x, d2.x), make_float2(d1.y, d2.y)},
                                 cpair{make_float2(e1.x, e2.x), make_float2(e1.y, e2.y)});
                        }
                    }
                    if (threadIdx.x == 0) emit(put, 0, folded(0), folded(h));
                } else {
                    for (int k0 = threadIdx.x; 2 * k0 <= h; k0 += U * blockDim.x) {
                        cpair xk[U], xh[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int k = k0 + u * blockDim.x;
                            if (2 * k <= h) {
                                xk[u] = folded(k);
                                xh[u] = folded(h - k);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int k = k0 + u * blockDim.x;
                            if (2 * k > h) break;
                            emit(put, k, xk[u], xh[u]);
                        }
                    }
                }
                if (blu)  // Bluestein zero padding
                    for (int k = h + threadIdx.x; k < M; k += blockDim.x)
                        put(k, cpair{make_float2(0.f, 0.f), make_float2(0.f, 0.f)});
                __syncthreads();
            };
            float2 *o1 = reinterpret_cast<float2 *>(a.map + (int64_t)b * a.npix + a.rd.poff[i]);
            float2 *o2 = reinterpret_cast<float2 *>(a.map + (int64_t)b * a.npix + a.rd.poff[i2]);
            // the last transform pass writes both rings straight to the maps: x_2q, x_2q+1
            auto st = [&](int q, cpair z) {
                if (q < h) {
                    if (blu) z = fft::e_mul(z, cscalef(chirp_at(chirp, q, h), inv_m));
                    o1[q] = make_float2(z.re.x, z.im.x);
                    if (pair) o2[q] = make_float2(z.re.y, z.im.y);
                }
            };
            if (blu) {
                // Bluestein takes natural order; the inverse chirp is the conjugate of the
                // forward one, and so is its spectrum (the chirp sequence is even)
                fill([&](int k, cpair v) { sm(k, v); });
                fft::convolve<L, true>(buf, a.tw, fb, sm, st);
            } else {
                // the adjoint transform wants digit-reversed input
                fill([&](int k, cpair v) { sm(fft::digitrev<L>(k), v); });
                fft::adj<L>(buf, a.tw, st);
            }
        }
    }
};

// Rings of n = 4q pixels too long for one Bluestein buffer (the transpose of the forward
// split), the ring pair packed as one complex sequence: the n folded coefficients X go to
// shared memory, the radix-4 step
//   Z_p[k'] = W_n^{-p k'} sum_t W_4^{-p t} X[k' + t q]
// runs in place, then four q-point inverse DFTs by Bluestein write pixels 4 s + p.
struct InvSplitCta {
    const FftInvArgs &a;
    float2 *buf, *X;
    const float2 *chirp, *fb;  // chirp exp(+i pi k^2 / q), k <= q/2
    int i, i2, n, hs;
    bool pair;
    float wsc;
    template <int L>
    __device__ void run()
    {
        const int q = n / 4;
        const float inv_m = 1.0f / (float)(1 << L);
        const int bend = min(a.B, (int)(blockIdx.y + 1) * a.mchunk);
        for (int b = blockIdx.y * a.mchunk; b < bend; ++b) {
            const float2 *c1 = a.c + ((int64_t)b * a.R + i) * a.NH;
            const float2 *c2 = a.c + ((int64_t)b * a.R + i2) * a.NH;
            for (int k = threadIdx.x; k < n; k += blockDim.x) {
                const bool up = 2 * k > n;
                const int mm = up ? n - k : k;
                const float2 ph = hs ? expipi_ratio(mm, n) : make_float2(1.f, 0.f);
                float2 d1 = folded_coeff(c1, mm, n, hs, ph, a.N, a.basic);
                float2 d2 = pair ? folded_coeff(c2, mm, n, hs, ph, a.N, a.basic) : make_float2(0.f, 0.f);
                if (up) {
                    d1.y = -d1.y;
                    d2.y = -d2.y;
                }
                X[k] = make_float2(wsc * (d1.x - d2.y), wsc * (d1.y + d2.x));
            }
            __syncthreads();
            for (int k = threadIdx.x; k < q; k += blockDim.x) {
                float2 v0 = X[k], v1 = X[q + k], v2 = X[2 * q + k], v3 = X[3 * q + k];
                fft::dft4<true>(v0, v1, v2, v3);
                const float2 w1 = expipi_ratio(2 * k, n), w2 = cmulf(w1, w1), w3 = cmulf(w1, w2);
                X[k] = v0;
                X[q + k] = cmulf(v1, w1);
                X[2 * q + k] = cmulf(v2, w2);
                X[3 * q + k] = cmulf(v3, w3);
            }
            __syncthreads();
            float *o1 = a.map + (int64_t)b * a.npix + a.rd.poff[i];
            float *o2 = a.map + (int64_t)b * a.npix + a.rd.poff[i2];
            for (int p = 0; p < 4; ++p) {
                const float2 *Z = X + p * q;
                auto ld = [&](int k) { return k < q ? cmulf(Z[k], chirp_at(chirp, k, q)) : make_float2(0.f, 0.f); };
                auto st = [&](int s, float2 z) {
                    if (s < q) {
                        z = cscalef(cmulf(z, chirp_at(chirp, s, q)), inv_m);
                        o1[4 * s + p] = z.x;
                        if (pair) o2[4 * s + p] = z.y;
                    }
                };
                fft::convolve<L, true>(buf, a.tw, fb, ld, st);
            }
        }
    }
};

__global__ void __launch_bounds__(512) k_fft_inv_split(FftInvArgs a)
{
    // [buffer_words(a.M)] quarter-transform buffer | [n] coefficients | chirp of the quarter
    extern __shared__ float2 sbuf[];
    ring::stage_allow_next();
    const int i = a.reps[blockIdx.x];
    if (a.skip_poles && i == 0) return;
    const int n = a.rd.n[i], q = n / 4;
    float2 *X = sbuf + fft::buffer_words(a.M);
    float2 *chirp = X + n;
    ring::chirp_table(chirp, q, +1);
    const int i2 = a.R - 1 - i;
    InvSplitCta c{a, sbuf, X, chirp, a.rd.fb + a.rd.fboff[i], i, i2, n, a.rd.hs[i], i2 != i,
                  a.weight ? a.rd.w[i] : 1.0f};
    c.run<13>();  // split rings have 2048 < q < 4096: quarter buffer 8192 (kMaxSplitM)
    ring::stage_wait_prev();
}

template <int LMAX>
__global__ void __launch_bounds__(ring::ClassShape<LMAX>::kThreads, ring::ClassShape<LMAX>::kMinBlocks)
k_fft_inv(FftInvArgs a)
{
    // [buffer_words(a.M)] pair buffer | short-ring fold: [2 (N/8 + 1)] folded coefficients,
    // [2 blockDim] float4 partial sums | chirp and phase tables
    extern __shared__ float4 smem4[];
    ring::stage_allow_next();
    const int i = a.reps[blockIdx.x];
    if (a.skip_poles && i == 0) return;  // rings 0 and R-1 come from the pole kernel
    const int n = a.rd.n[i], h = n / 2;
    const bool blu = ring::bluestein(h);
    const int logM = ring::log2_buffer(h);
    const int hs = a.rd.hs[i];
    const bool stage = a.stage_c && !a.basic && 4 * n < a.N;
    cpair *buf = reinterpret_cast<cpair *>(smem4);
    float2 *D1 = reinterpret_cast<float2 *>(buf + fft::buffer_words(a.M)), *D2 = D1 + (a.N / 8 + 1);
    float4 *part = reinterpret_cast<float4 *>(D2 + (a.N / 8 + 1));
    float2 *chirp = a.stage_c ? reinterpret_cast<float2 *>(part + 2 * blockDim.x) : D1;  // exp(+i pi k^2 / h)
    float2 *phase = chirp + (blu ? h / 2 + 1 : 0);                                    // exp(+i pi m / n)
    ring::tables(chirp, phase, n, h, +1, blu, a.tw);
    const int i2 = a.R - 1 - i;
    InvCta c{a, buf, D1, D2, part, chirp, phase, blu ? a.rd.fb + a.rd.fboff[i] : nullptr,
             i, i2, n, h, hs, i2 != i, blu, stage, a.weight ? a.rd.w[i] : 1.0f};
    ring::dispatch_upto<LMAX>(logM, c);
    ring::stage_wait_prev();
}

}  // namespace

// Shared memory of a ring FFT class: the transform buffer (pairs of complex values, or single
// ones for the split path), the short-ring fold's bins and partial sums, and the per-ring
// tables.
size_t fft_smem_bytes(int M, int N, bool stage_c, int tab, int threads, bool split)
{
    size_t bytes = (size_t)fft::buffer_words(M) * (split ? sizeof(float2) : sizeof(cpair));
    size_t words = (size_t)tab;
    if (stage_c) words += 2 * (size_t)(N / 8 + 1) + 4 * (size_t)threads;
    return bytes + words * sizeof(float2);
}

cudaError_t launch_fft_inv_split(const FftInvArgs &a, int count, int threads, cudaStream_t st, bool after_prev)
{
    if (count <= 0) return cudaSuccess;
    const size_t smem = fft_smem_bytes(a.M, a.N, false, a.tab, threads, true);
    cudaError_t e = cudaFuncSetAttribute((const void *)k_fft_inv_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return launch_class_kernel(k_fft_inv_split, dim3(count, (a.B + a.mchunk - 1) / a.mchunk), threads, smem, st,
                               after_prev, a);
}

template <int LMAX>
cudaError_t launch_inv_class(const FftInvArgs &a, int count, cudaStream_t st, bool after_prev)
{
    constexpr int T = ring::ClassShape<LMAX>::kThreads;
    const size_t smem = fft_smem_bytes(a.M, a.N, a.stage_c != 0, a.tab, T, false);
    cudaError_t e = cudaFuncSetAttribute((const void *)k_fft_inv<LMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return launch_class_kernel(k_fft_inv<LMAX>, dim3(count, (a.B + a.mchunk - 1) / a.mchunk), T, smem, st,
                               after_prev, a);
}

cudaError_t launch_fft_inv(const FftInvArgs &a, int count, int threads, cudaStream_t st, bool after_prev)
{
    (void)threads;  // the class's own launch shape (ring_common.cuh ClassShape)
    if (count <= 0) return cudaSuccess;
    if (a.logM <= 10) return launch_inv_class<10>(a, count, st, after_prev);
    if (a.logM == 11) return launch_inv_class<11>(a, count, st, after_prev);
    if (a.logM == 12) return launch_inv_class<12>(a, count, st, after_prev);
    return launch_inv_class<13>(a, count, st, after_prev);
}

}  // namespace arkcos
