// Batched mixed-length ring FFTs (Sec. 4.1: real-to-complex FFT of every ring, length 4i in
// the polar caps and 4 nside on the equatorial belt; the inverse after the ring-band sum).
//
// One CTA owns one ring pair (j, R-1-j): mirror rings have the same length and offset, so
// their two real rings are packed as the real and imaginary parts of one complex sequence
// and split afterwards by Hermitian symmetry.  The CTA loops over all maps of the batch.
// Transforms run in shared memory over a power-of-two buffer M (fft_engine.cuh: radix-16
// passes in registers, padded shared memory):
//   - power-of-two rings (M = n): one forward DIF transform (digit-reversed spectrum) or,
//     on the inverse side, the adjoint transform from digit-reversed input;
//   - other lengths: Bluestein's chirp-z algorithm (1970) with M >= 2n - 1: DIF of the
//     chirped sequence, pointwise product with the chirp spectrum held in registers (computed
//     once per CTA) fused with the last DIF and first adjoint pass, adjoint back to natural
//     order -- no explicit digit-reversal pass.
// The chirps and first-pixel phases of a ring are tabulated once per CTA in shared memory
// (the chirp only up to n/2: chirp(n - k) = (-1)^n chirp(k)) and reused by every map.
// Epilogues fold in the first-pixel phase exp(-i m phi0) (Eq. fftrot), the ring weight and,
// on the inverse side, the Sec. 4.3 fold of super-Nyquist modes.
#include "fft_engine.cuh"

namespace arkcos {

namespace {


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
__device__ void ring_tables(float2 *chirp, float2 *phase, int n, bool blu, bool hs, int sgn)
{
    if (blu)
        for (int k = threadIdx.x; 2 * k <= n; k += blockDim.x) chirp[k] = expipi_ratio(sgn * k * k, n);
    if (hs)
        for (int m = threadIdx.x; m <= n / 2; m += blockDim.x) phase[m] = expipi_ratio(sgn * m, n);
    __syncthreads();
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

// DIF spectrum (digit-reversed positions) of the Bluestein sequence b_k = exp(+i pi k^2 / n),
// |k| < n, circular in M, of every Bluestein ring of a class: computed once per grid.
__global__ void __launch_bounds__(1024) k_chirp_spectra(FftFwdArgs a, float2 *fb_all)
{
    extern __shared__ float2 buf[];
    const int j = a.reps[blockIdx.x];
    const int n = a.rd.n[j];
    const int logM = ring_log2_buffer(n);
    const int M = 1 << logM;
    if (M == n) return;  // power-of-two ring: no chirp
    auto ld = [&](int k) {
        int kk = -1;
        if (k < n) kk = k;
        else if (k > M - n) kk = M - k;
        return kk < 0 ? make_float2(0.f, 0.f) : expipi_ratio(kk * kk, n);
    };
    fft::dif(buf, logM, a.tw, ld);
    const fft::Smem sm{buf, fft::top_shift(logM)};
    float2 *fb = fb_all + a.rd.fboff[j];
    for (int p = threadIdx.x; p < M; p += blockDim.x) fb[p] = sm(p);
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
    float2 *chirp = buf + fft::buffer_words(a.M);   // exp(-i pi k^2 / n), k <= n/2
    float2 *phase = chirp + (blu ? n / 2 + 1 : 0);  // exp(-i pi m / n)
    ring_tables(chirp, phase, n, blu, hs, -1);
    const float2 *fb = blu ? a.rd.fb + a.rd.fboff[j] : nullptr;
    const float wsc = a.weight ? a.rd.w[j] : 1.0f;
    const bool zero = a.zero_poles && j == 0;
    const float inv_m = 1.0f / (float)M;
    const fft::Smem sm{buf, fft::top_shift(logM)};
    for (int b = 0; b < a.B; ++b) {
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
        if (blu) fft::convolve<false>(buf, logM, a.tw, fb, ld, sm);
        else fft::dif(buf, logM, a.tw, ld);
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
                    zm = cscalef(cmulf(sm(mb), chirp_at(chirp, mb, n)), inv_m);
                    zn = cscalef(cmulf(sm(mn), chirp_at(chirp, mn, n)), inv_m);
                } else {
                    zm = sm(fft::digitrev(mb, logM));
                    zn = sm(fft::digitrev(mn, logM));
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
                zm = cscalef(cmulf(sm(m), chirp_at(chirp, m, n)), inv_m);
                zn = cscalef(cmulf(sm(mn), chirp_at(chirp, mn, n)), inv_m);
            } else {
                zm = sm(fft::digitrev(m, logM));
                zn = sm(fft::digitrev(mn, logM));
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
    float2 *cs1 = buf + fft::buffer_words(a.M), *cs2 = cs1 + a.NH;
    float2 *chirp = cs1 + (a.stage_c ? 2 * a.NH : 0);  // exp(+i pi k^2 / n), k <= n/2
    float2 *phase = chirp + (blu ? n / 2 + 1 : 0);      // exp(+i pi m / n)
    ring_tables(chirp, phase, n, blu, hs, +1);
    const float2 *fb = blu ? a.rd.fb + a.rd.fboff[i] : nullptr;
    const float wsc = a.weight ? a.rd.w[i] : 1.0f;
    const float inv_m = 1.0f / (float)M;
    const fft::Smem sm{buf, fft::top_shift(logM)};
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
        // ring values of frequency k: X = D(i) + i D(i2), folded (Sec. 4.3) and weighted
        auto coeff = [&](int k) {
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
                v = make_float2(wsc * (d1.x - d2.y), wsc * (d1.y + d2.x));
                if (blu) v = cmulf(v, chirp_at(chirp, k, n));
            }
            return v;
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
            // forward one, and so is its spectrum (the chirp sequence is even).  The first pass
            // computes the coefficients itself when it keeps every thread busy and no ring
            // folds many modes; otherwise all threads stage them first.
            if (!stage && M >= 16 * (int)blockDim.x) {
                fft::convolve<true>(buf, logM, a.tw, fb, coeff, st);
            } else {
                for (int k = threadIdx.x; k < M; k += blockDim.x) sm(k, coeff(k));
                __syncthreads();
                fft::convolve<true>(buf, logM, a.tw, fb, sm, st);
            }
        } else {
            // the adjoint transform wants digit-reversed input
            for (int k = threadIdx.x; k < M; k += blockDim.x) sm(fft::digitrev(k, logM), coeff(k));
            __syncthreads();
            fft::adj(buf, logM, a.tw, st);
        }
        __syncthreads();
    }
}

}  // namespace

size_t fft_smem_bytes(int M, int N, bool stage_c, int tab)
{
    size_t words = (size_t)fft::buffer_words(M) + (size_t)tab;
    if (stage_c) words += 2 * (size_t)(N / 2 + 1);
    return words * sizeof(float2);
}

static cudaError_t set_smem(const void *fn, size_t bytes)
{
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
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
