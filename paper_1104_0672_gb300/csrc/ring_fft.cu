// Batched mixed-length ring FFTs (Sec. 4.1: real-to-complex FFT of every ring, length 4i in
// the polar caps and 4 nside on the equatorial belt; the inverse after the ring-band sum).
//
// One CTA owns one ring pair (j, R-1-j): mirror rings have the same length and offset, so
// their two real rings are packed as the real and imaginary parts of one complex sequence
// and split afterwards by Hermitian symmetry.  The transform runs in shared memory:
// radix-2 Cooley-Tukey for power-of-two lengths and Bluestein's chirp-z algorithm (1970)
// over a power-of-two buffer for every other length.  The CTA loops over all maps of the
// batch, so the Bluestein chirp spectrum is computed once per ring pair and kept in
// registers.  Epilogues fold in the first-pixel phase exp(-i m phi0) (Eq. fftrot), the
// ring weight and, on the inverse side, the Sec. 4.3 fold of super-Nyquist modes.
#include "device_common.cuh"

namespace arkcos {

namespace {

constexpr int kFbPer = 16;  // chirp-spectrum elements per thread (M <= 16 * blockDim)

__device__ __forceinline__ int brev(int e, int logM)
{
    return (int)(__brev((unsigned)e) >> (32 - logM));
}

// In-place radix-2 decimation in time: bit-reversed input, natural-order output.
__device__ void fft_dit(float2 *x, int M, const float2 *__restrict__ tw, bool inv)
{
    const int half = M >> 1;
    for (int h = 1; h < M; h <<= 1) {
        for (int b = threadIdx.x; b < half; b += blockDim.x) {
            const int pos = b & (h - 1);
            const int i0 = ((b - pos) << 1) + pos, i1 = i0 + h;
            float2 w = __ldg(&tw[h + pos]);
            if (inv) w.y = -w.y;
            const float2 u = x[i0], v = cmulf(x[i1], w);
            x[i0] = caddf(u, v);
            x[i1] = csubf(u, v);
        }
        __syncthreads();
    }
}

// In-place radix-2 decimation in frequency: natural-order input, bit-reversed output.
__device__ void fft_dif(float2 *x, int M, const float2 *__restrict__ tw, bool inv)
{
    const int half = M >> 1;
    for (int h = half; h >= 1; h >>= 1) {
        for (int b = threadIdx.x; b < half; b += blockDim.x) {
            const int pos = b & (h - 1);
            const int i0 = ((b - pos) << 1) + pos, i1 = i0 + h;
            float2 w = __ldg(&tw[h + pos]);
            if (inv) w.y = -w.y;
            const float2 u = x[i0], v = x[i1];
            x[i0] = caddf(u, v);
            x[i1] = cmulf(csubf(u, v), w);
        }
        __syncthreads();
    }
}

__device__ void bitrev_permute(float2 *x, int M, int logM)
{
    for (int e = threadIdx.x; e < M; e += blockDim.x) {
        const int r = brev(e, logM);
        if (e < r) {
            const float2 t = x[e];
            x[e] = x[r];
            x[r] = t;
        }
    }
    __syncthreads();
}

// Spectrum of the Bluestein chirp b_k = exp(sgn i pi k^2 / n), |k| < n, circular in M;
// element e = tid + r * blockDim of the natural-order result lands in fb[r].
__device__ void chirp_spectrum(float2 *buf, int M, int logM, int n, int sgn,
                               const float2 *__restrict__ tw, float2 (&fb)[kFbPer])
{
    for (int e = threadIdx.x; e < M; e += blockDim.x) {
        const int k = brev(e, logM);
        int kk = -1;
        if (k < n) kk = k;
        else if (k > M - n) kk = M - k;
        buf[e] = kk < 0 ? make_float2(0.f, 0.f) : expipi_ratio(sgn * (long long)kk * kk, n);
    }
    __syncthreads();
    fft_dit(buf, M, tw, false);
#pragma unroll
    for (int r = 0; r < kFbPer; ++r) {
        const int e = threadIdx.x + r * blockDim.x;
        fb[r] = e < M ? buf[e] : make_float2(0.f, 0.f);
    }
    __syncthreads();
}

// Convolution step of Bluestein: buf holds DIT(a) (natural order); multiply by the chirp
// spectrum and transform back.  Result conv[m] sits at buf[brev(m)], scaled by M.
__device__ void bluestein_finish(float2 *buf, int M, const float2 *__restrict__ tw,
                                 const float2 (&fb)[kFbPer])
{
#pragma unroll
    for (int r = 0; r < kFbPer; ++r) {
        const int e = threadIdx.x + r * blockDim.x;
        if (e < M) buf[e] = cmulf(buf[e], fb[r]);
    }
    __syncthreads();
    fft_dif(buf, M, tw, true);
}

__global__ void __launch_bounds__(1024) k_fft_fwd(FftFwdArgs a)
{
    extern __shared__ float2 buf[];
    const int j = a.reps[blockIdx.x];
    const int j2 = a.R - 1 - j;
    const bool pair = j2 != j;
    const int n = a.rd.n[j];
    const int M = a.M, logM = a.logM;
    const bool blu = (M != n);
    float2 fb[kFbPer];
    if (blu) chirp_spectrum(buf, M, logM, n, +1, a.tw, fb);
    const float wsc = a.weight ? a.rd.w[j] : 1.0f;
    const int hs = a.rd.hs[j];
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
                if (blu) v = cmulf(v, expipi_ratio(-(long long)k * k, n));
            }
            buf[k] = v;
        }
        __syncthreads();
        bitrev_permute(buf, M, logM);
        fft_dit(buf, M, a.tw, false);
        if (blu) bluestein_finish(buf, M, a.tw, fb);
        float2 *s1 = a.spec + (int64_t)b * a.nspec + a.rd.soff[j];
        float2 *s2 = a.spec + (int64_t)b * a.nspec + a.rd.soff[j2];
        for (int m = threadIdx.x; m <= n / 2; m += blockDim.x) {
            const int mn = m == 0 ? 0 : n - m;
            float2 zm, zn;
            if (blu) {
                zm = cscalef(cmulf(buf[brev(m, logM)], expipi_ratio(-(long long)m * m, n)), inv_m);
                zn = cscalef(cmulf(buf[brev(mn, logM)], expipi_ratio(-(long long)mn * mn, n)), inv_m);
            } else {
                zm = buf[m];
                zn = buf[mn];
            }
            const float2 ph = hs ? expipi_ratio(-(long long)m, n) : make_float2(1.f, 0.f);
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
__device__ __forceinline__ float2 folded_coeff(const float2 *__restrict__ c, int mm, int n, int hs,
                                               int NH, int N, bool basic)
{
    float2 acc = make_float2(0.f, 0.f);
    const int nyq = N / 2;
    if (basic) {
        float2 d = c[mm];
        if (hs) d = cmulf(d, expipi_ratio(mm, n));
        if (2 * mm == n) d.y = 0.f;  // (d + conj d) / 2
        return d;
    }
    for (int m = mm; m <= nyq; m += n) {
        float2 d = __ldg(&c[m]);
        if (hs) d = cmulf(d, expipi_ratio(m, n));
        const float h = (m == nyq) ? 0.5f : 1.0f;
        acc.x += h * d.x;
        acc.y += h * d.y;
    }
    for (int m = n - mm; m <= nyq; m += n) {
        if (m == 0) continue;
        float2 d = __ldg(&c[m]);
        if (hs) d = cmulf(d, expipi_ratio(m, n));
        const float h = (m == nyq) ? 0.5f : 1.0f;
        acc.x += h * d.x;
        acc.y -= h * d.y;
    }
    (void)NH;
    return acc;
}

__global__ void __launch_bounds__(1024) k_fft_inv(FftInvArgs a)
{
    extern __shared__ float2 buf[];
    const int i = a.reps[blockIdx.x];
    if (a.skip_poles && i == 0) return;  // rings 0 and R-1 come from the pole kernel
    const int i2 = a.R - 1 - i;
    const bool pair = i2 != i;
    const int n = a.rd.n[i];
    const int M = a.M, logM = a.logM;
    const bool blu = (M != n);
    float2 fb[kFbPer];
    if (blu) chirp_spectrum(buf, M, logM, n, -1, a.tw, fb);
    const float wsc = a.weight ? a.rd.w[i] : 1.0f;
    const int hs = a.rd.hs[i];
    const float inv_m = 1.0f / (float)M;
    for (int b = 0; b < a.B; ++b) {
        const float2 *c1 = a.c + ((int64_t)b * a.R + i) * a.NH;
        const float2 *c2 = a.c + ((int64_t)b * a.R + i2) * a.NH;
        for (int k = threadIdx.x; k < M; k += blockDim.x) {
            float2 v = make_float2(0.f, 0.f);
            if (k < n) {
                const bool up = 2 * k > n;
                const int mm = up ? n - k : k;
                float2 d1 = folded_coeff(c1, mm, n, hs, a.NH, a.N, a.basic);
                float2 d2 = pair ? folded_coeff(c2, mm, n, hs, a.NH, a.N, a.basic)
                                 : make_float2(0.f, 0.f);
                if (up) {
                    d1.y = -d1.y;
                    d2.y = -d2.y;
                }
                // X = D(i) + i D(i2)
                v = make_float2(wsc * (d1.x - d2.y), wsc * (d1.y + d2.x));
                if (blu) v = cmulf(v, expipi_ratio((long long)k * k, n));
            }
            buf[k] = v;
        }
        __syncthreads();
        bitrev_permute(buf, M, logM);
        fft_dit(buf, M, a.tw, !blu);
        if (blu) bluestein_finish(buf, M, a.tw, fb);
        float *o1 = a.map + (int64_t)b * a.npix + a.rd.poff[i];
        float *o2 = a.map + (int64_t)b * a.npix + a.rd.poff[i2];
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            float2 z;
            if (blu)
                z = cscalef(cmulf(buf[brev(p, logM)], expipi_ratio((long long)p * p, n)), inv_m);
            else
                z = buf[p];
            o1[p] = z.x;
            if (pair) o2[p] = z.y;
        }
        __syncthreads();
    }
}

}  // namespace

static cudaError_t set_smem(const void *fn, size_t bytes)
{
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_fft_fwd(const FftFwdArgs &a, int count, int threads, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const size_t smem = (size_t)a.M * sizeof(float2);
    cudaError_t e = set_smem((const void *)k_fft_fwd, smem);
    if (e != cudaSuccess) return e;
    k_fft_fwd<<<count, threads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fft_inv(const FftInvArgs &a, int count, int threads, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const size_t smem = (size_t)a.M * sizeof(float2);
    cudaError_t e = set_smem((const void *)k_fft_inv, smem);
    if (e != cudaSuccess) return e;
    k_fft_inv<<<count, threads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace arkcos
