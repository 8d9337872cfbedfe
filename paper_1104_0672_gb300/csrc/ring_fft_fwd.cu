// Forward ring transforms (Sec. 4.1: real-to-complex FFT of every ring, length 4i in the
// polar caps and 4 nside on the equatorial belt) and the per-grid Bluestein chirp spectra.
// The epilogue folds in the first-pixel phase exp(-i m phi0) (Eq. fftrot) and the ring weight
// and writes either the half spectra or, for the ring-band contraction, the extended spectra
// of ring and mirror over every kernel-grid mode (Sec. 4.3).
#include <algorithm>

#include "ring_common.cuh"

namespace arkcos {

namespace {

using ring::chirp_at;

// DIF spectrum (digit-reversed positions) of the Bluestein sequence b_k = exp(+i pi k^2 / n),
// |k| < n, circular in M, of every Bluestein ring of a class: computed once per grid.
struct ChirpCta {
    float2 *buf, *fb;
    const float2 *tw;
    int n;
    template <int L>
    __device__ void run()
    {
        constexpr int M = 1 << L;
        const int nn = n;
        auto ld = [&](int k) {
            int kk = -1;
            if (k < nn) kk = k;
            else if (k > M - nn) kk = M - k;
            return kk < 0 ? make_float2(0.f, 0.f) : expipi_ratio(kk * kk, nn);
        };
        fft::dif<L>(buf, tw, ld);
        const fft::Smem<L> sm{buf};
        for (int p = threadIdx.x; p < M; p += blockDim.x) fb[p] = sm(p);
    }
};

__global__ void __launch_bounds__(1024) k_chirp_spectra(FftFwdArgs a, float2 *fb_all)
{
    extern __shared__ float2 buf[];
    const int j = a.reps[blockIdx.x];
    const int n = a.split ? a.rd.n[j] / 4 : a.rd.n[j];  // split rings: the chirp of the quarter
    const int logM = ring::log2_buffer(n);
    if ((1 << logM) == n) return;  // power-of-two ring: no chirp
    ChirpCta c{buf, fb_all + a.rd.fboff[j], a.tw, n};
    ring::dispatch(logM, c);
}

struct FwdCta {
    const FftFwdArgs &a;
    float2 *buf;
    const float2 *chirp, *phase, *fb;
    int j, j2, n, hs;
    bool pair, blu, zero;
    float wsc;

    // exp(-i m phi0) for m <= n/2: the table, or computed when the ring has none (split rings)
    __device__ __forceinline__ float2 phase_at(int m) const
    {
        if (!hs) return make_float2(1.f, 0.f);
        return phase ? phase[m] : expipi_ratio(-m, n);
    }

    // Output for map b from the ring-pair spectrum Z_f = z(f), f in [0, n).
    template <bool POW2, int L, class Z>
    __device__ __forceinline__ void epilogue(int b, Z z) const
    {
        const int nn = POW2 ? (1 << L) : n;
        if (a.ext4) {
            // every kernel-grid mode m <= N/2: the periodic extension a_{m + qn} =
            // exp(-i q n phi0) a_m (ENHANCED) or the Nyquist-halved truncation (BASIC)
            float4 *o4 = a.spec4 + ((int64_t)b * a.nrep + j) * a.NH;
            for (int m = threadIdx.x; m < a.NH; m += blockDim.x) {
                int q, mm;
                if (POW2) {
                    q = m >> L;
                    mm = m & (nn - 1);
                } else {
                    q = (int)__fdividef((float)m, (float)nn);
                    mm = m - q * nn;
                    if (mm < 0) {
                        --q;
                        mm += nn;
                    } else if (mm >= nn) {
                        ++q;
                        mm -= nn;
                    }
                }
                const bool up = 2 * mm > nn;
                const int mb = up ? nn - mm : mm;  // base mode in [0, n/2]
                const int mn = mb == 0 ? 0 : nn - mb;
                const float2 zm = z(mb), zn = z(mn);
                const float2 ph = phase_at(mb);
                float2 ea = cmulf(make_float2(0.5f * (zm.x + zn.x), 0.5f * (zm.y - zn.y)), ph);
                // the middle ring is its own mirror: its row holds (a, a)
                float2 eb = pair ? cmulf(make_float2(0.5f * (zm.y + zn.y), -0.5f * (zm.x - zn.x)), ph)
                                 : ea;
                float sc = wsc;
                if (a.basic) {
                    if (q > 0 || up) sc = 0.f;
                    else if (2 * mm == nn && nn < a.N) sc *= 0.5f;
                } else {
                    if (up) {
                        ea.y = -ea.y;
                        eb.y = -eb.y;
                    }
                    if (hs && ((q + (up ? 1 : 0)) & 1)) sc = -sc;
                }
                o4[m] = make_float4(sc * ea.x, sc * ea.y, sc * eb.x, sc * eb.y);
            }
        } else {
            float2 *s1 = a.spec + (int64_t)b * a.nspec + a.rd.soff[j];
            float2 *s2 = a.spec + (int64_t)b * a.nspec + a.rd.soff[j2];
            for (int m = threadIdx.x; m <= nn / 2; m += blockDim.x) {
                const int mn = m == 0 ? 0 : nn - m;
                const float2 zm = z(m), zn = z(mn);
                const float2 ph = phase_at(m);
                const float2 ea = make_float2(0.5f * (zm.x + zn.x), 0.5f * (zm.y - zn.y));
                s1[m] = cscalef(cmulf(ea, ph), wsc);
                if (pair) {
                    // (Z_m - conj Z_{n-m}) / (2i)
                    const float2 eb = make_float2(0.5f * (zm.y + zn.y), -0.5f * (zm.x - zn.x));
                    s2[m] = cscalef(cmulf(eb, ph), wsc);
                }
            }
        }
        __syncthreads();
    }

    template <int L>
    __device__ void run()
    {
        const fft::Smem<L> sm{buf};
        const float inv_m = 1.0f / (float)(1 << L);
        const int bend = min(a.B, (int)(blockIdx.y + 1) * a.mchunk);
        for (int b = blockIdx.y * a.mchunk; b < bend; ++b) {
            const float *m1 = a.map + (int64_t)b * a.npix + a.rd.poff[j];
            const float *m2 = a.map + (int64_t)b * a.npix + a.rd.poff[j2];
            // the first transform pass reads the ring pair straight from the maps
            auto ld = [&](int k) {
                float2 v = make_float2(0.f, 0.f);
                if (k < n && !zero) {
                    v.x = __ldg(&m1[k]);
                    v.y = pair ? __ldg(&m2[k]) : 0.f;
                    if (blu) v = cmulf(v, chirp_at(chirp, k, n));
                }
                return v;
            };
            if (blu) {
                fft::convolve<L, false>(buf, a.tw, fb, ld, sm);
                epilogue<false, L>(b, [&](int f) { return cscalef(cmulf(sm(f), chirp_at(chirp, f, n)), inv_m); });
            } else {
                fft::dif<L>(buf, a.tw, ld);
                epilogue<true, L>(b, [&](int f) { return sm(fft::digitrev<L>(f)); });
            }
        }
    }
};

// Rings of n = 4q pixels too long for one Bluestein buffer: decimation in time by 4,
//   X[k' + t q] = sum_p W_n^{p k'} W_4^{p t} Y_p[k'],   Y_p = DFT_q(z[4 s + p]),
// with the four q-point DFTs by Bluestein one after the other into the spectrum area X of
// shared memory, then the radix-4 combination in place.
struct FwdSplitCta {
    FwdCta &f;
    float2 *X;  // [n] spectrum area
    template <int L>
    __device__ void run()
    {
        const FftFwdArgs &a = f.a;
        const int n = f.n, q = n / 4;
        const float inv_m = 1.0f / (float)(1 << L);
        const float2 *chq = f.chirp;  // exp(-i pi k^2 / q), k <= q/2
        const int bend = min(a.B, (int)(blockIdx.y + 1) * a.mchunk);
        for (int b = blockIdx.y * a.mchunk; b < bend; ++b) {
            const float *m1 = a.map + (int64_t)b * a.npix + a.rd.poff[f.j];
            const float *m2 = a.map + (int64_t)b * a.npix + a.rd.poff[f.j2];
            for (int p = 0; p < 4; ++p) {
                auto ld = [&](int s) {
                    float2 v = make_float2(0.f, 0.f);
                    if (s < q && !f.zero) {
                        v.x = __ldg(&m1[4 * s + p]);
                        v.y = f.pair ? __ldg(&m2[4 * s + p]) : 0.f;
                        v = cmulf(v, chirp_at(chq, s, q));
                    }
                    return v;
                };
                float2 *Y = X + p * q;
                auto st = [&](int s, float2 v) {
                    if (s < q) Y[s] = cscalef(cmulf(v, chirp_at(chq, s, q)), inv_m);
                };
                fft::convolve<L, false>(f.buf, a.tw, f.fb, ld, st);
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
            f.template epilogue<false, L>(b, [&](int k) { return X[k]; });
        }
    }
};

__global__ void __launch_bounds__(1024) k_fft_fwd_split(FftFwdArgs a)
{
    // [buffer_words(a.M)] quarter-transform buffer | [n] spectrum | chirp of the quarter
    extern __shared__ float2 buf[];
    const int j = a.reps[blockIdx.x];
    const int n = a.rd.n[j], q = n / 4;
    const int hs = a.rd.hs[j];
    float2 *X = buf + fft::buffer_words(a.M);
    float2 *chirp = X + n;
    ring::tables(chirp, nullptr, q, true, false, -1);
    const int j2 = a.R - 1 - j;
    FwdCta c{a, buf, chirp, nullptr, a.rd.fb + a.rd.fboff[j], j, j2, n, hs,
             j2 != j, true, a.zero_poles && j == 0, a.weight ? a.rd.w[j] : 1.0f};
    FwdSplitCta sc{c, X};
    sc.run<13>();  // split rings have 2048 < q < 4096: quarter buffer 8192 (kMaxSplitM)
}

__global__ void __launch_bounds__(1024) k_fft_fwd(FftFwdArgs a)
{
    extern __shared__ float2 buf[];  // [buffer_words(a.M)] transform buffer, then the tables
    const int j = a.reps[blockIdx.x];
    const int n = a.rd.n[j];
    const int logM = ring::log2_buffer(n);  // a launch may cover several buffer sizes <= a.M
    const bool blu = (1 << logM) != n;
    const int hs = a.rd.hs[j];
    float2 *chirp = buf + fft::buffer_words(a.M);   // exp(-i pi k^2 / n), k <= n/2
    float2 *phase = chirp + (blu ? n / 2 + 1 : 0);  // exp(-i pi m / n)
    ring::tables(chirp, phase, n, blu, hs, -1);
    const int j2 = a.R - 1 - j;
    FwdCta c{a, buf, chirp, phase, blu ? a.rd.fb + a.rd.fboff[j] : nullptr, j, j2, n, hs,
             j2 != j, blu, a.zero_poles && j == 0, a.weight ? a.rd.w[j] : 1.0f};
    ring::dispatch(logM, c);
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

cudaError_t launch_fft_fwd_split(const FftFwdArgs &a, int count, int threads, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const size_t smem = fft_smem_bytes(a.M, a.N, false, a.tab, threads);
    cudaError_t e = set_smem((const void *)k_fft_fwd_split, smem);
    if (e != cudaSuccess) return e;
    k_fft_fwd_split<<<dim3(count, (a.B + a.mchunk - 1) / a.mchunk), threads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fft_fwd(const FftFwdArgs &a, int count, int threads, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const size_t smem = fft_smem_bytes(a.M, a.N, false, a.tab, threads);
    cudaError_t e = set_smem((const void *)k_fft_fwd, smem);
    if (e != cudaSuccess) return e;
    k_fft_fwd<<<dim3(count, (a.B + a.mchunk - 1) / a.mchunk), threads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace arkcos
