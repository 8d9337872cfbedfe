// Inverse ring transforms after the ring-band sum (Sec. 4.1), with the Sec. 4.3 fold of the
// kernel-grid modes onto each ring's own frequencies.
#include "ring_common.cuh"

namespace arkcos {

namespace {

using ring::chirp_at;

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

// The same fold for every mm of a short ring pair with the whole CTA: thread (mm, chunk)
// sums the aliases t = chunk, chunk + C, ... of bin mm for both rings, then each bin adds its
// C partial sums (part: 2 C (n/2 + 1) <= 2 blockDim entries) in chunk order.  c1, c2 are the
// staged coefficients of rings i and i2.
__device__ __forceinline__ void fold_all(const float2 *c1, const float2 *c2, bool pair, int n, int hs,
                                         const float2 *phase, int N, float2 *D1, float2 *D2, float4 *part)
{
    const int nh = n / 2 + 1, nyq = N / 2, T = blockDim.x;
    int C = 1;
    while (2 * C * nh <= T) C *= 2;
    for (int w = threadIdx.x; w < nh * C; w += T) {
        const int mm = w / C, ch = w - mm * C;
        float2 p1 = make_float2(0.f, 0.f), p2 = p1, q1 = p1, q2 = p1;
        // positive aliases m = mm + t n: weight (-1)^t with the offset, 1/2 at the Nyquist mode
        for (int t = ch;; t += C) {
            const int m = mm + t * n;
            if (m > nyq) break;
            const float h = (m == nyq ? 0.5f : 1.0f) * ((hs && (t & 1)) ? -1.f : 1.f);
            float2 d1 = c1[m], d2 = c2[m];
            if (m == 0) d1.y = d2.y = 0.f;  // the m = 0 term of a real ring
            p1.x += h * d1.x;
            p1.y += h * d1.y;
            p2.x += h * d2.x;
            p2.y += h * d2.y;
        }
        // negative aliases -m, m = t n - mm, t >= 1
        for (int t = 1 + ch;; t += C) {
            const int m = t * n - mm;
            if (m > nyq) break;
            const float h = (m == nyq ? 0.5f : 1.0f) * ((hs && (t & 1)) ? -1.f : 1.f);
            const float2 d1 = c1[m], d2 = c2[m];
            q1.x += h * d1.x;
            q1.y += h * d1.y;
            q2.x += h * d2.x;
            q2.y += h * d2.y;
        }
        if (C == 1) {  // one thread per bin: finish it here
            const float2 ph = hs ? phase[mm] : make_float2(1.f, 0.f);
            const float2 a1 = cmulf(p1, ph), g1 = cmulf(q1, cconjf(ph));
            const float2 a2 = cmulf(p2, ph), g2 = cmulf(q2, cconjf(ph));
            D1[mm] = make_float2(a1.x + g1.x, a1.y - g1.y);
            D2[mm] = pair ? make_float2(a2.x + g2.x, a2.y - g2.y) : make_float2(0.f, 0.f);
        } else {       // nh C <= blockDim partial sums
            part[2 * w] = make_float4(p1.x, p1.y, q1.x, q1.y);
            part[2 * w + 1] = make_float4(p2.x, p2.y, q2.x, q2.y);
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
        const float2 ph = hs ? phase[mm] : make_float2(1.f, 0.f);
        float2 a1 = cmulf(make_float2(s1.x, s1.y), ph), g1 = cmulf(make_float2(s1.z, s1.w), cconjf(ph));
        float2 a2 = cmulf(make_float2(s2.x, s2.y), ph), g2 = cmulf(make_float2(s2.z, s2.w), cconjf(ph));
        D1[mm] = make_float2(a1.x + g1.x, a1.y - g1.y);
        D2[mm] = pair ? make_float2(a2.x + g2.x, a2.y - g2.y) : make_float2(0.f, 0.f);
    }
    __syncthreads();
}

struct InvCta {
    const FftInvArgs &a;
    float2 *buf, *cs1, *cs2, *D1, *D2;
    float4 *part;
    const float2 *chirp, *phase, *fb;
    int i, i2, n, hs;
    bool pair, blu, stage;
    float wsc;

    template <int L>
    __device__ void run()
    {
        constexpr int M = 1 << L;
        const fft::Smem<L> sm{buf};
        const float inv_m = 1.0f / (float)M;
        const int bend = min(a.B, (int)(blockIdx.y + 1) * a.mchunk);
        for (int b = blockIdx.y * a.mchunk; b < bend; ++b) {
            const float2 *c1 = a.c + ((int64_t)b * a.R + i) * a.NH;
            const float2 *c2 = a.c + ((int64_t)b * a.R + i2) * a.NH;
            if (stage) {
                // short rings fold many modes onto each frequency: stage the coefficients with
                // coalesced loads, then fold them with the whole CTA
                constexpr int U = 8;  // loads in flight per thread
                for (int m0 = threadIdx.x; m0 < a.NH; m0 += U * blockDim.x) {
                    float2 v1[U], v2[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int m = m0 + u * blockDim.x;
                        v1[u] = m < a.NH ? __ldg(&c1[m]) : make_float2(0.f, 0.f);
                        v2[u] = (pair && m < a.NH) ? __ldg(&c2[m]) : make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int m = m0 + u * blockDim.x;
                        if (m < a.NH) {
                            cs1[m] = v1[u];
                            cs2[m] = v2[u];
                        }
                    }
                }
                __syncthreads();
                fold_all(cs1, cs2, pair, n, hs, phase, a.N, D1, D2, part);
            }
            // the folded coefficients D(mm) of ring and mirror, mm in [0, n/2]
            auto folded = [&](int mm, float2 &d1, float2 &d2) {
                if (stage) {
                    d1 = D1[mm];
                    d2 = D2[mm];
                } else {
                    const float2 ph = hs ? phase[mm] : make_float2(1.f, 0.f);
                    d1 = folded_coeff(c1, mm, n, hs, ph, a.N, a.basic);
                    d2 = pair ? folded_coeff(c2, mm, n, hs, ph, a.N, a.basic) : make_float2(0.f, 0.f);
                }
            };
            // transform input at frequencies mm and n - mm from one evaluation of D(mm):
            // X_k = D_k(i) + i D_k(i2) with D_{n-k} = conj D_k, weighted (and chirped)
            auto emit = [&](auto put, int mm, float2 d1, float2 d2) {
                float2 v = make_float2(wsc * (d1.x - d2.y), wsc * (d1.y + d2.x));
                float2 w = make_float2(wsc * (d1.x + d2.y), wsc * (d2.x - d1.y));  // conj'd D
                if (blu) {
                    const float2 ch = chirp_at(chirp, mm, n);
                    v = cmulf(v, ch);
                    // chirp(n - mm) = (-1)^n chirp(mm)
                    w = cmulf(w, (n & 1) ? make_float2(-ch.x, -ch.y) : ch);
                }
                put(mm, v);
                if (mm > 0 && 2 * mm < n) put(n - mm, w);
            };
            auto fill = [&](auto put) {
                const int nyq = a.N / 2;
                if (!stage && !a.basic && 2 * n > a.N) {
                    // rings longer than N/2 have at most one alias on each side (m = mm and
                    // m = n - mm): the loads of four frequencies are issued together
                    constexpr int U = 4;
                    for (int m0 = threadIdx.x; 2 * m0 <= n; m0 += U * blockDim.x) {
                        float2 p1[U], p2[U], q1[U], q2[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int mm = m0 + u * blockDim.x, mn = n - mm;
                            const bool ok = 2 * mm <= n, neg = ok && mn <= nyq;
                            p1[u] = ok ? __ldg(&c1[mm]) : make_float2(0.f, 0.f);
                            p2[u] = ok && pair ? __ldg(&c2[mm]) : make_float2(0.f, 0.f);
                            q1[u] = neg ? __ldg(&c1[mn]) : make_float2(0.f, 0.f);
                            q2[u] = neg && pair ? __ldg(&c2[mn]) : make_float2(0.f, 0.f);
                        }
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int mm = m0 + u * blockDim.x, mn = n - mm;
                            if (2 * mm > n) break;
                            // the fold of folded_coeff with its two terms written out
                            const float2 ph = hs ? phase[mm] : make_float2(1.f, 0.f);
                            const float hp = mm == nyq ? 0.5f : 1.0f;
                            const float hq = (mn == nyq ? 0.5f : 1.0f) * (hs ? -1.f : 1.f);
                            float2 x1 = p1[u], x2 = p2[u];
                            if (mm == 0) x1.y = x2.y = 0.f;  // the m = 0 term of a real ring
                            float2 d1 = cmulf(cscalef(x1, hp), ph), d2 = cmulf(cscalef(x2, hp), ph);
                            const float2 g1 = cmulf(cscalef(q1[u], hq), cconjf(ph));
                            const float2 g2 = cmulf(cscalef(q2[u], hq), cconjf(ph));
                            d1 = make_float2(d1.x + g1.x, d1.y - g1.y);
                            d2 = make_float2(d2.x + g2.x, d2.y - g2.y);
                            emit(put, mm, d1, d2);
                        }
                    }
                } else {
                    for (int mm = threadIdx.x; 2 * mm <= n; mm += blockDim.x) {
                        float2 d1, d2;
                        folded(mm, d1, d2);
                        emit(put, mm, d1, d2);
                    }
                }
                if (blu)  // Bluestein zero padding
                    for (int k = n + threadIdx.x; k < M; k += blockDim.x) put(k, make_float2(0.f, 0.f));
                __syncthreads();
            };
            float *o1 = a.map + (int64_t)b * a.npix + a.rd.poff[i];
            float *o2 = a.map + (int64_t)b * a.npix + a.rd.poff[i2];
            // the last transform pass writes the ring pair straight to the maps
            auto st = [&](int p, float2 z) {
                if (p < n) {
                    if (blu) z = cscalef(cmulf(z, chirp_at(chirp, p, n)), inv_m);
                    o1[p] = z.x;
                    if (pair) o2[p] = z.y;
                }
            };
            if (blu) {
                // Bluestein takes natural order; the inverse chirp is the conjugate of the
                // forward one, and so is its spectrum (the chirp sequence is even)
                fill([&](int k, float2 v) { sm(k, v); });
                fft::convolve<L, true>(buf, a.tw, fb, sm, st);
            } else {
                // the adjoint transform wants digit-reversed input
                fill([&](int k, float2 v) { sm(fft::digitrev<L>(k), v); });
                fft::adj<L>(buf, a.tw, st);
            }
        }
    }
};

// Rings of n = 4q pixels too long for one Bluestein buffer (the transpose of the forward
// split): the n folded coefficients X go to shared memory, the radix-4 step
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

__global__ void __launch_bounds__(1024) k_fft_inv_split(FftInvArgs a)
{
    // [buffer_words(a.M)] quarter-transform buffer | [n] coefficients | chirp of the quarter
    extern __shared__ float2 buf[];
    const int i = a.reps[blockIdx.x];
    if (a.skip_poles && i == 0) return;
    const int n = a.rd.n[i], q = n / 4;
    float2 *X = buf + fft::buffer_words(a.M);
    float2 *chirp = X + n;
    ring::tables(chirp, nullptr, q, true, false, +1);
    const int i2 = a.R - 1 - i;
    InvSplitCta c{a, buf, X, chirp, a.rd.fb + a.rd.fboff[i], i, i2, n, a.rd.hs[i], i2 != i,
                  a.weight ? a.rd.w[i] : 1.0f};
    c.run<13>();  // split rings have 2048 < q < 4096: quarter buffer 8192 (kMaxSplitM)
}

__global__ void __launch_bounds__(1024) k_fft_inv(FftInvArgs a)
{
    // [buffer_words(a.M)] buffer | staging: [2 NH] coefficients, [2 (N/8 + 1)] folded
    // coefficients, [2 blockDim] float4 partial sums | chirp and phase tables
    extern __shared__ float2 buf[];
    const int i = a.reps[blockIdx.x];
    if (a.skip_poles && i == 0) return;  // rings 0 and R-1 come from the pole kernel
    const int n = a.rd.n[i];
    const int logM = ring::log2_buffer(n);
    const bool blu = (1 << logM) != n;
    const int hs = a.rd.hs[i];
    const bool stage = a.stage_c && !a.basic && 4 * n < a.N;
    float2 *cs1 = buf + fft::buffer_words(a.M), *cs2 = cs1 + a.NH;
    float2 *D1 = cs2 + a.NH, *D2 = D1 + (a.N / 8 + 1);
    float4 *part = reinterpret_cast<float4 *>(D2 + (a.N / 8 + 1));
    float2 *chirp = a.stage_c ? reinterpret_cast<float2 *>(part + 2 * blockDim.x) : cs1;  // exp(+i pi k^2 / n)
    float2 *phase = chirp + (blu ? n / 2 + 1 : 0);                                        // exp(+i pi m / n)
    ring::tables(chirp, phase, n, blu, hs, +1);
    const int i2 = a.R - 1 - i;
    InvCta c{a, buf, cs1, cs2, D1, D2, part, chirp, phase, blu ? a.rd.fb + a.rd.fboff[i] : nullptr,
             i, i2, n, hs, i2 != i, blu, stage, a.weight ? a.rd.w[i] : 1.0f};
    ring::dispatch(logM, c);
}

}  // namespace

size_t fft_smem_bytes(int M, int N, bool stage_c, int tab, int threads)
{
    size_t words = (size_t)fft::buffer_words(M) + (size_t)tab;
    if (stage_c) words += 2 * (size_t)(N / 2 + 1) + 2 * (size_t)(N / 8 + 1) + 4 * (size_t)threads;
    return words * sizeof(float2);
}

cudaError_t launch_fft_inv_split(const FftInvArgs &a, int count, int threads, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const size_t smem = fft_smem_bytes(a.M, a.N, false, a.tab, threads);
    cudaError_t e = cudaFuncSetAttribute((const void *)k_fft_inv_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_fft_inv_split<<<dim3(count, (a.B + a.mchunk - 1) / a.mchunk), threads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fft_inv(const FftInvArgs &a, int count, int threads, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const size_t smem = fft_smem_bytes(a.M, a.N, a.stage_c != 0, a.tab, threads);
    cudaError_t e = cudaFuncSetAttribute((const void *)k_fft_inv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_fft_inv<<<dim3(count, (a.B + a.mchunk - 1) / a.mchunk), threads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace arkcos
