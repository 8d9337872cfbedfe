// Forward ring transforms (Sec. 4.1: real-to-complex FFT of every ring, length 4i in the
// polar caps and 4 nside on the equatorial belt) and the per-grid Bluestein chirp spectra.
// The epilogue folds in the first-pixel phase exp(-i m phi0) (Eq. fftrot) and the ring weight
// and writes either the half spectra or, for the ring-band contraction, the extended spectra
// of ring and mirror over every kernel-grid mode (Sec. 4.3).
#include <algorithm>

#include "ring_common.cuh"

namespace arkcos {

namespace {

using fft::cpair;
using ring::chirp_at;

// DIF spectrum (digit-reversed positions) of the Bluestein sequence b_k = exp(+i pi k^2 / l),
// |k| < l, circular in M, for the l-point transform of every Bluestein ring of a class
// (l = n/2, or n/4 for split rings): computed once per grid.
struct ChirpCta {
    float2 *buf, *fb;
    const float2 *tw;
    int l;
    template <int L>
    __device__ void run()
    {
        constexpr int M = 1 << L;
        const int ll = l;
        auto ld = [&](int k) {
            int kk = -1;
            if (k < ll) kk = k;
            else if (k > M - ll) kk = M - k;
            return kk < 0 ? make_float2(0.f, 0.f) : expipi_ratio(kk * kk, ll);
        };
        fft::dif<L>(buf, tw, ld);
        const fft::Smem<L> sm{buf};
        for (int p = threadIdx.x; p < M; p += blockDim.x) fb[p] = sm(p);
    }
};

__global__ void __launch_bounds__(512) k_chirp_spectra(FftFwdArgs a, float2 *fb_all)
{
    extern __shared__ float2 buf[];
    const int j = a.reps[blockIdx.x];
    const int l = a.split ? a.rd.n[j] / 4 : a.rd.n[j] / 2;
    if (!ring::bluestein(l)) return;  // power-of-two transform: no chirp
    ChirpCta c{buf, fb_all + a.rd.fboff[j], a.tw, l};
    ring::dispatch(ring::log2_buffer(l), c);
}

// One ring pair through the h-point transforms of its two rings (lanes of a cpair).
struct FwdCta {
    const FftFwdArgs &a;
    cpair *buf;
    cpair *xh;                    // shared slot of X_h (the Nyquist term) in the two-phase epilogue
    const float2 *chirp, *phase;  // chirp of h (Bluestein rings), exp(-i pi m / n) for m <= n/2
    const float2 *fb;
    int j, j2, n, h, hs;
    bool pair, blu, zero;
    float wsc;

    // exp(-i pi m / n), 0 <= m <= n/2
    __device__ __forceinline__ float2 ph(int m) const { return phase[m]; }

    // X_k and X_{h-k} of both rings from Z_k and Z_{h-k} (Z_h = Z_0), each times the first-pixel
    // phase and the ring weight:
    //   X_k = E + w O,  X_{h-k} = conj(E - w O),  E = (Z_k + conj Z_{h-k}) / 2,
    //   O = -i (Z_k - conj Z_{h-k}) / 2,  w = exp(-2 pi i k / n)
    __device__ __forceinline__ void split(const cpair &zk, const cpair &zh, int k, cpair &xk, cpair &xhk) const
    {
        using namespace fft;
        const float2 Er = pmul(bcast(0.5f), caddf(zk.re, zh.re)), Ei = pmul(bcast(0.5f), csubf(zk.im, zh.im));
        const float2 Or = pmul(bcast(0.5f), caddf(zk.im, zh.im)), Oi = pmul(bcast(-0.5f), csubf(zk.re, zh.re));
        const float2 w = ph(2 * k);
        const float2 Wr = pfma(Oi, bcast(-w.y), pmul(Or, bcast(w.x)));
        const float2 Wi = pfma(Or, bcast(w.y), pmul(Oi, bcast(w.x)));
        const cpair a0{caddf(Er, Wr), caddf(Ei, Wi)}, a1{csubf(Er, Wr), csubf(Wi, Ei)};
        const float2 p0 = hs ? ph(k) : make_float2(1.f, 0.f), p1 = hs ? ph(h - k) : make_float2(1.f, 0.f);
        xk = e_mul(a0, cscalef(p0, wsc));
        xhk = e_mul(a1, cscalef(p1, wsc));
    }

    // both rings' values as (ring j, ring j2); the middle ring is its own mirror: (a, a)
    __device__ __forceinline__ float4 out4(const cpair &x) const
    {
        const float4 v = ring::lanes4(x);
        return pair ? v : make_float4(v.x, v.y, v.x, v.y);
    }

    // Output for map b from the h-point spectra Z_k = z(k), k < h (natural order), whose
    // shared-memory slot is pos(k).
    template <int L, class Z, class Pos>
    __device__ __forceinline__ void epilogue(int b, Z z, Pos pos) const
    {
        const int hh = h;
        if (!a.ext4) {
            // half spectra of the two rings, m = 0..n/2
            float2 *s1 = a.spec + (int64_t)b * a.nspec + a.rd.soff[j];
            float2 *s2 = a.spec + (int64_t)b * a.nspec + a.rd.soff[j2];
            for (int k = threadIdx.x; 2 * k <= hh; k += blockDim.x) {
                cpair xk, xhk;
                split(z(k), z(k == 0 ? 0 : hh - k), k, xk, xhk);
                const float4 u = ring::lanes4(xk), v = ring::lanes4(xhk);
                s1[k] = make_float2(u.x, u.y);
                if (pair) s2[k] = make_float2(u.z, u.w);
                if (2 * k != hh) {  // X_{h/2} is its own partner
                    s1[hh - k] = make_float2(v.x, v.y);
                    if (pair) s2[hh - k] = make_float2(v.z, v.w);
                }
            }
            __syncthreads();
            return;
        }
        float4 *o4 = a.spec4 + ((int64_t)b * a.nrep + j) * a.NH;
        if (n == a.N) {
            // every kernel-grid mode m <= N/2 = h is one of the ring's own: X_m directly
            for (int k = threadIdx.x; 2 * k <= hh; k += blockDim.x) {
                cpair xk, xhk;
                split(z(k), z(k == 0 ? 0 : hh - k), k, xk, xhk);
                o4[k] = out4(xk);
                if (2 * k != hh) o4[hh - k] = out4(xhk);
            }
            __syncthreads();
            return;
        }
        // shorter rings: X_m (m <= h) in place, then every kernel-grid mode m <= N/2 from it:
        // the periodic extension a_{m + qn} = exp(-i q n phi0) a_m (ENHANCED) or the
        // Nyquist-halved truncation (BASIC)
        for (int k = threadIdx.x; 2 * k <= hh; k += blockDim.x) {
            // each thread owns the two slots it reads, so X overwrites Z in place
            cpair xk, xhk;
            split(z(k), z(k == 0 ? 0 : hh - k), k, xk, xhk);
            buf[fft::Geo<L>::sp(pos(k))] = xk;
            if (k == 0) *xh = xhk;
            else if (2 * k != hh) buf[fft::Geo<L>::sp(pos(hh - k))] = xhk;
        }
        __syncthreads();
        const int nn = n;
        for (int m = threadIdx.x; m < a.NH; m += blockDim.x) {
            int q = (int)__fdividef((float)m, (float)nn);
            int mm = m - q * nn;
            if (mm < 0) {
                --q;
                mm += nn;
            } else if (mm >= nn) {
                ++q;
                mm -= nn;
            }
            const bool up = 2 * mm > nn;
            const int mb = up ? nn - mm : mm;  // base mode in [0, n/2]
            const float4 v = out4(mb == hh ? *xh : buf[fft::Geo<L>::sp(pos(mb))]);
            float sc = 1.f;
            float4 r = v;
            if (a.basic) {
                if (q > 0 || up) sc = 0.f;
                else if (2 * mm == nn && nn < a.N) sc = 0.5f;
            } else {
                if (up) {
                    r.y = -r.y;
                    r.w = -r.w;
                }
                if (hs && ((q + (up ? 1 : 0)) & 1)) sc = -1.f;
            }
            o4[m] = make_float4(sc * r.x, sc * r.y, sc * r.z, sc * r.w);
        }
        __syncthreads();
    }

    template <int L>
    __device__ void run()
    {
        constexpr int M = 1 << L;
        const fft::Smem<L, cpair> sm{buf};
        const float inv_m = 1.0f / (float)M;
        const int bend = min(a.B, (int)(blockIdx.y + 1) * a.mchunk);
        for (int b = blockIdx.y * a.mchunk; b < bend; ++b) {
            const float2 *m1 = reinterpret_cast<const float2 *>(a.map + (int64_t)b * a.npix + a.rd.poff[j]);
            const float2 *m2 = reinterpret_cast<const float2 *>(a.map + (int64_t)b * a.npix + a.rd.poff[j2]);
            if (b + 1 < bend) {
                // the next map's pixels of both rings into L2 while this map is transformed
                const char *p1 = reinterpret_cast<const char *>(m1 + a.npix / 2);
                const char *p2 = reinterpret_cast<const char *>(m2 + a.npix / 2);
                const int lines = (n * 4 + 127) / 128;
                for (int l = threadIdx.x; l < 2 * lines; l += blockDim.x)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"((l < lines ? p1 : p2) + 128 * (l % lines)));
            }
            // the first transform pass reads both rings straight from the maps: z_q = x_2q + i x_2q+1
            auto ld = [&](int q) {
                cpair v{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
                if (q < h && !zero) {
                    const float2 u = __ldg(&m1[q]);
                    const float2 w = pair ? __ldg(&m2[q]) : make_float2(0.f, 0.f);
                    v = cpair{make_float2(u.x, w.x), make_float2(u.y, w.y)};
                    if (blu) v = fft::e_mul(v, chirp_at(chirp, q, h));
                }
                return v;
            };
            if (blu) {
                fft::convolve<L, false>(buf, a.tw, fb, ld, sm);
                epilogue<L>(
                    b, [&](int k) { return fft::e_mul(sm(k), cscalef(chirp_at(chirp, k, h), inv_m)); },
                    [](int k) { return k; });
            } else {
                fft::dif<L>(buf, a.tw, ld);
                epilogue<L>(b, [&](int k) { return sm(fft::digitrev<L>(k)); }, [](int k) { return fft::digitrev<L>(k); });
            }
        }
    }
};

// Rings of n = 4q pixels too long for one Bluestein buffer: decimation in time by 4,
//   X[k' + t q] = sum_p W_n^{p k'} W_4^{p t} Y_p[k'],   Y_p = DFT_q(z[4 s + p]),
// with the ring pair packed as one complex sequence z = x_j + i x_j2, the four q-point DFTs by
// Bluestein one after the other into the spectrum area X of shared memory, then the radix-4
// combination in place and the split of the two rings.
struct FwdSplitCta {
    const FftFwdArgs &a;
    float2 *buf, *X;
    const float2 *chirp, *fb;  // chirp exp(-i pi k^2 / q), k <= q/2
    int j, j2, n, hs;
    bool pair, zero;
    float wsc;

    __device__ __forceinline__ float2 phase_at(int m) const
    {
        return hs ? expipi_ratio(-m, n) : make_float2(1.f, 0.f);
    }

    template <int L>
    __device__ void run()
    {
        const int q = n / 4;
        const float inv_m = 1.0f / (float)(1 << L);
        const int bend = min(a.B, (int)(blockIdx.y + 1) * a.mchunk);
        for (int b = blockIdx.y * a.mchunk; b < bend; ++b) {
            const float *m1 = a.map + (int64_t)b * a.npix + a.rd.poff[j];
            const float *m2 = a.map + (int64_t)b * a.npix + a.rd.poff[j2];
            for (int p = 0; p < 4; ++p) {
                auto ld = [&](int s) {
                    float2 v = make_float2(0.f, 0.f);
                    if (s < q && !zero) {
                        v.x = __ldg(&m1[4 * s + p]);
                        v.y = pair ? __ldg(&m2[4 * s + p]) : 0.f;
                        v = cmulf(v, chirp_at(chirp, s, q));
                    }
                    return v;
                };
                float2 *Y = X + p * q;
                auto st = [&](int s, float2 v) {
                    if (s < q) Y[s] = cscalef(cmulf(v, chirp_at(chirp, s, q)), inv_m);
                };
                fft::convolve<L, false>(buf, a.tw, fb, ld, st);
            }
            for (int k = threadIdx.x; k < q; k += blockDim.x) {
                float2 y0 = X[k], y1 = X[q + k], y2 = X[2 * q + k], y3 = X[3 * q + k];
                const float2 w1 = expipi_ratio(-2 * k, n), w2 = cmulf(w1, w1), w3 = cmulf(w1, w2);
                y1 = cmulf(y1, w1);
                y2 = cmulf(y2, w2);
                y3 = cmulf(y3, w3);
                fft::dft4<false>(y0, y1, y2, y3);
                X[k] = y0;
                X[q + k] = y1;
                X[2 * q + k] = y2;
                X[3 * q + k] = y3;
            }
            __syncthreads();
            // split of the packed ring pair, phase, weight and the extension (as FwdCta)
            if (!a.ext4) {
                float2 *s1 = a.spec + (int64_t)b * a.nspec + a.rd.soff[j];
                float2 *s2 = a.spec + (int64_t)b * a.nspec + a.rd.soff[j2];
                for (int m = threadIdx.x; m <= n / 2; m += blockDim.x) {
                    const int mn = m == 0 ? 0 : n - m;
                    const float2 zm = X[m], zn = X[mn];
                    const float2 ph = phase_at(m);
                    s1[m] = cscalef(cmulf(make_float2(0.5f * (zm.x + zn.x), 0.5f * (zm.y - zn.y)), ph), wsc);
                    if (pair) s2[m] = cscalef(cmulf(make_float2(0.5f * (zm.y + zn.y), -0.5f * (zm.x - zn.x)), ph), wsc);
                }
            } else {
                float4 *o4 = a.spec4 + ((int64_t)b * a.nrep + j) * a.NH;
                for (int m = threadIdx.x; m < a.NH; m += blockDim.x) {
                    const int qq = m / n, mm = m - qq * n;
                    const bool up = 2 * mm > n;
                    const int mb = up ? n - mm : mm;
                    const int mn = mb == 0 ? 0 : n - mb;
                    const float2 zm = X[mb], zn = X[mn];
                    const float2 ph = phase_at(mb);
                    float2 ea = cmulf(make_float2(0.5f * (zm.x + zn.x), 0.5f * (zm.y - zn.y)), ph);
                    float2 eb = pair ? cmulf(make_float2(0.5f * (zm.y + zn.y), -0.5f * (zm.x - zn.x)), ph) : ea;
                    float sc = wsc;
                    if (a.basic) {
                        if (qq > 0 || up) sc = 0.f;
                        else if (2 * mm == n && n < a.N) sc *= 0.5f;
                    } else {
                        if (up) {
                            ea.y = -ea.y;
                            eb.y = -eb.y;
                        }
                        if (hs && ((qq + (up ? 1 : 0)) & 1)) sc = -sc;
                    }
                    o4[m] = make_float4(sc * ea.x, sc * ea.y, sc * eb.x, sc * eb.y);
                }
            }
            __syncthreads();
        }
    }
};

__global__ void __launch_bounds__(512) k_fft_fwd_split(FftFwdArgs a)
{
    // [buffer_words(a.M)] quarter-transform buffer | [n] spectrum | chirp of the quarter
    extern __shared__ float2 sbuf[];
    ring::stage_allow_next();
    const int j = a.reps[blockIdx.x];
    const int n = a.rd.n[j], q = n / 4;
    float2 *X = sbuf + fft::buffer_words(a.M);
    float2 *chirp = X + n;
    ring::chirp_table(chirp, q, -1);
    const int j2 = a.R - 1 - j;
    FwdSplitCta c{a, sbuf, X, chirp, a.rd.fb + a.rd.fboff[j], j, j2, n, a.rd.hs[j], j2 != j,
                  a.zero_poles && j == 0, a.weight ? a.rd.w[j] : 1.0f};
    c.run<13>();  // split rings have 2048 < q < 4096: quarter buffer 8192 (kMaxSplitM)
    ring::stage_wait_prev();
}

template <int LMAX>
__global__ void __launch_bounds__(ring::ClassShape<LMAX>::kThreads, ring::ClassShape<LMAX>::kMinBlocks)
k_fft_fwd(FftFwdArgs a)
{
    // [buffer_words(a.M)] pair buffer, then the chirp and phase tables of Bluestein rings
    extern __shared__ float4 smem4[];
    __shared__ cpair xh;
    ring::stage_allow_next();
    const int j = a.reps[blockIdx.x];
    const int n = a.rd.n[j], h = n / 2;
    const bool blu = ring::bluestein(h);
    const int logM = ring::log2_buffer(h);  // a launch may cover several buffer sizes <= a.M
    const int hs = a.rd.hs[j];
    cpair *buf = reinterpret_cast<cpair *>(smem4);
    float2 *chirp = reinterpret_cast<float2 *>(buf + fft::buffer_words(a.M));  // exp(-i pi k^2 / h)
    float2 *phase = chirp + (blu ? h / 2 + 1 : 0);                              // exp(-i pi m / n)
    ring::tables(chirp, phase, n, h, -1, blu, a.tw);
    const int j2 = a.R - 1 - j;
    FwdCta c{a, buf, &xh, chirp, phase, blu ? a.rd.fb + a.rd.fboff[j] : nullptr, j, j2, n, h, hs,
             j2 != j, blu, a.zero_poles && j == 0, a.weight ? a.rd.w[j] : 1.0f};
    ring::dispatch_upto<LMAX>(logM, c);
    ring::stage_wait_prev();
}

cudaError_t set_smem(const void *fn, size_t bytes)
{
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

// Classes of few ring pairs (the short rings) split their maps over several CTAs so that the
// launch still fills the GPU; large classes keep every map of a ring pair in one CTA, which
// computes the ring's tables once.  split_mult (from the autotuner) multiplies the splits.
int fft_map_chunk(int count, int nmaps, int split_mult)
{
    const int splits = std::max(1, std::min(nmaps, std::max(1, 2048 / std::max(count, 1)) * std::max(split_mult, 1)));
    return (nmaps + splits - 1) / splits;
}

cudaError_t launch_chirp_spectra(const FftFwdArgs &a, float2 *fb, int count, int threads, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const size_t smem = (size_t)fft::buffer_words(a.M) * sizeof(float2);
    cudaError_t e = set_smem((const void *)k_chirp_spectra, smem);
    if (e != cudaSuccess) return e;
    k_chirp_spectra<<<count, threads, smem, st>>>(a, fb);
    return cudaGetLastError();
}

cudaError_t launch_fft_fwd_split(const FftFwdArgs &a, int count, int threads, cudaStream_t st, bool after_prev)
{
    if (count <= 0) return cudaSuccess;
    const size_t smem = fft_smem_bytes(a.M, a.N, false, a.tab, threads, true);
    cudaError_t e = set_smem((const void *)k_fft_fwd_split, smem);
    if (e != cudaSuccess) return e;
    return launch_class_kernel(k_fft_fwd_split, dim3(count, (a.B + a.mchunk - 1) / a.mchunk), threads, smem, st,
                               after_prev, a);
}

template <int LMAX>
cudaError_t launch_fwd_class(const FftFwdArgs &a, int count, cudaStream_t st, bool after_prev)
{
    constexpr int T = ring::ClassShape<LMAX>::kThreads;
    const size_t smem = fft_smem_bytes(a.M, a.N, false, a.tab, T, false);
    cudaError_t e = set_smem((const void *)k_fft_fwd<LMAX>, smem);
    if (e != cudaSuccess) return e;
    return launch_class_kernel(k_fft_fwd<LMAX>, dim3(count, (a.B + a.mchunk - 1) / a.mchunk), T, smem, st,
                               after_prev, a);
}

cudaError_t launch_fft_fwd(const FftFwdArgs &a, int count, int threads, cudaStream_t st, bool after_prev)
{
    (void)threads;  // the class's own launch shape (ring_common.cuh ClassShape)
    if (count <= 0) return cudaSuccess;
    if (a.logM <= 10) return launch_fwd_class<10>(a, count, st, after_prev);
    if (a.logM == 11) return launch_fwd_class<11>(a, count, st, after_prev);
    if (a.logM == 12) return launch_fwd_class<12>(a, count, st, after_prev);
    return launch_fwd_class<13>(a, count, st, after_prev);
}

}  // namespace arkcos
