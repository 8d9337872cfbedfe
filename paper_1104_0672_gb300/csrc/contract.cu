// Kernel sampling and the ring-band contraction (Sec. 4.1: kernel grid centred on each output
// ring, its ring FFT, product with the map coefficients and the sum over the n_support rings
// in theta; Sec. 4.3: super-Nyquist periodic extension and the equatorial shift fix).
//
// The kernel grid of ring pair (i, j) is sampled at longitudes x_k = pi (2k + f) / N with
// f = 1 when the shift fix applies to a pair of equal-length rings with different offsets
// (delta = +-pi/N) and f = 0 otherwise.  The samples are symmetric about x = 0, so the
// pair's Fourier coefficient including the offset phase is real:
//     rho_m(i,j) = sum_{k >= 0} c_k K(u(x_k)) cos(m x_k),   c_k = multiplicity(k) / N,
// and the contraction is c_m(i) = sum_j rho_m(i,j) w_j a_m(j) (w_j folded into a).
//
// k_taps evaluates c_k K(u) per pair in FP64 (u is the squared chord of Eq. kernel_angle
// in the cancellation-free form 4[B cos^2(x/2) + A sin^2(x/2)]), storing FP32 values.
// k_contract generates rho for a block of output rings x 128 modes into shared memory (one
// thread per mode, cosines by Reinsch's modified recurrence, restarted from exact values
// every 64 taps) and then contracts it with the map spectra of every map of the batch.
// N-S mirror pairs share rho, so each CTA serves ring i and ring R-1-i.
#include <algorithm>

#include "fft_engine.cuh"

namespace arkcos {

namespace {

constexpr int kRingBlock = 8;   // representative output rings per CTA
constexpr int kMapGroups = 4;   // warp groups per CTA: they split the coefficient generation
                                // by pairs and the contraction by maps

// Kernel samples K(u(x_k)) c_k / N.  u = 4 (B cos^2(x/2) + A sin^2(x/2)) is the haversine form
// of the squared chord, so the FP64 work per sample is the offset from the knot below it,
// u - u_t = 4B c2 + 4A s2 - u_t (two FMAs); the knot segment comes from an FP32 estimate of u
// (next to a knot the neighbouring segment's line differs by rounding only, the profile being
// continuous there) and the linear step runs in FP32 on tables pre-scaled by 1 / N.
__global__ void __launch_bounds__(256) k_taps(TapArgs a)
{
    extern __shared__ double tsm[];
    const int T = a.kd.T;
    double *ut = tsm;                                  // [T] knots in u
    float *utf = reinterpret_cast<float *>(tsm + T);   // [T] the same in FP32
    float *f = utf + T, *slope = f + T, *span = slope + T;  // [T] profile / N, its slope, knot spacing
    const double invN = 1.0 / (double)a.N;
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        ut[t] = a.kd.ut[t];
        utf[t] = (float)a.kd.ut[t];
        f[t] = (float)(a.kd.knots[t] * invN);
        if (t < T - 1) {
            const double du = a.kd.ut[t + 1] - a.kd.ut[t];
            slope[t] = (float)((a.kd.knots[t + 1] - a.kd.knots[t]) / du * invN);
            span[t] = (float)du;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const float umaxf = (float)a.kd.umax;
    for (int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < a.kd.npairs; p += warps) {
        const int fl = a.shift_fix ? a.kd.fl[p] : 0;
        const int S = fl ? a.kd.S1[p] : a.kd.S0[p];
        const int t0 = a.kd.toff[p], t1 = a.kd.toff[p + 1];
        const double A4 = 4.0 * a.kd.A[p], B4 = 4.0 * a.kd.B[p];
        const float A4f = (float)A4, B4f = (float)B4;
        for (int k = lane; k < t1 - t0; k += 32) {
            float val = 0.f;
            if (k <= S) {
                const int t = 2 * k + fl;  // x_k / 2 = pi t / (2N)
                const float uf = fminf(fmaf(B4f, a.s2f[a.N - t], A4f * a.s2f[t]), umaxf);
                const int sg = knot_segment_f(uf, utf, T, a.kd.gscale);
                const double d = fma(B4, a.s2[a.N - t], fma(A4, a.s2[t], -ut[sg]));
                // u is clamped to u_max: the last segment ends at its knot
                const float df = fminf((float)d, span[sg]);
                const float K = fmaf(df, slope[sg], f[sg]);
                val = (fl == 0 && (k == 0 || 2 * k == a.N)) ? K : 2.f * K;
            }
            a.taps[t0 + k] = val;
        }
    }
}


template <int H>
__global__ void __launch_bounds__(kModeBlock *kMapGroups) k_contract(ContractArgs a)
{
    extern __shared__ float rho[];  // [pair_chunk][kModeBlock]
    const int tid = threadIdx.x & (kModeBlock - 1);
    const int grp = threadIdx.x / kModeBlock;
    const int m = blockIdx.x * kModeBlock + tid;
    const bool mv = m < a.NH;
    const int r0 = blockIdx.y * H;
    const int nr = min(H, a.nrep - r0);
    const int b0 = blockIdx.z * a.maps_per_chunk;
    const int b1 = min(a.B, b0 + a.maps_per_chunk);
    const int kid = a.per_map ? (b0 - a.map_base) : 0;
    const KernDev &kd = a.kd[kid];
    const float *taps = a.taps[kid];

    int jlo[H], jhi[H], ps[H];
#pragma unroll
    for (int li = 0; li < H; ++li) {
        if (li < nr) {
            jlo[li] = kd.jlo[r0 + li];
            jhi[li] = kd.jhi[r0 + li];
            ps[li] = kd.pstart[r0 + li];
        } else {
            jlo[li] = 1;
            jhi[li] = 0;
            ps[li] = 0;
        }
    }
    const int P0 = kd.pstart[r0], P1 = kd.pstart[r0 + nr];
    const int ju0 = jlo[0];
    int ju1 = jhi[0];
#pragma unroll
    for (int li = 1; li < H; ++li) ju1 = max(ju1, jhi[li]);

    for (int c0 = P0; c0 < P1; c0 += a.pair_chunk) {
        const int c1 = min(P1, c0 + a.pair_chunk);
        // ---- generation: rho for pairs [c0, c1), this thread's mode, pairs split by group
        for (int p = c0 + grp; p < c1; p += kMapGroups) {
            const int f = a.shift_fix ? kd.fl[p] : 0;
            const int S = f ? kd.S1[p] : kd.S0[p];
            const float4 *tp4 = reinterpret_cast<const float4 *>(taps + kd.toff[p]);
            rho[(p - c0) * kModeBlock + tid] = mv ? gen_rho(tp4, S, f, m, a.N) : 0.f;
        }
        __syncthreads();
        // ---- contraction over the input rings of the band, maps split by group
        if (mv) {
            for (int b = b0 + grp; b < b1; b += kMapGroups) {
                const float4 *sp4b = map_spec4(a, b);
                float2 acc[H], acc2[H];
#pragma unroll
                for (int li = 0; li < H; ++li) {
                    if (c0 == P0 || li >= nr) {
                        acc[li] = make_float2(0.f, 0.f);
                        acc2[li] = make_float2(0.f, 0.f);
                    } else {
                        const int i = r0 + li;
                        acc[li] = a.c[((int64_t)b * a.R + i) * a.NH + m];
                        acc2[li] = a.c[((int64_t)b * a.R + (a.R - 1 - i)) * a.NH + m];
                    }
                }
                for (int j = ju0; j <= ju1; ++j) {
                    // skip rings no pair of this chunk uses
                    bool used = false;
#pragma unroll
                    for (int li = 0; li < H; ++li) {
                        const int p = ps[li] + j - jlo[li];
                        used |= (j >= jlo[li] && j <= jhi[li] && p >= c0 && p < c1);
                    }
                    if (!used) continue;
                    const float4 v = paired_coeff(sp4b, j, a.R, a.NH, m);
                    const float2 aj = make_float2(v.x, v.y), ajm = make_float2(v.z, v.w);
#pragma unroll
                    for (int li = 0; li < H; ++li) {
                        const int p = ps[li] + j - jlo[li];
                        if (j >= jlo[li] && j <= jhi[li] && p >= c0 && p < c1) {
                            const float r = rho[(p - c0) * kModeBlock + tid];
                            acc[li].x = fmaf(r, aj.x, acc[li].x);
                            acc[li].y = fmaf(r, aj.y, acc[li].y);
                            acc2[li].x = fmaf(r, ajm.x, acc2[li].x);
                            acc2[li].y = fmaf(r, ajm.y, acc2[li].y);
                        }
                    }
                }
#pragma unroll
                for (int li = 0; li < H; ++li) {
                    if (li < nr) {
                        const int i = r0 + li, im = a.R - 1 - i;
                        a.c[((int64_t)b * a.R + i) * a.NH + m] = acc[li];
                        if (im != i) a.c[((int64_t)b * a.R + im) * a.NH + m] = acc2[li];
                    }
                }
            }
        }
        __syncthreads();
    }
}

// Fast path of the contraction for bands of at most kBand2 input rings per output ring.
// Thread = (mode m, representative output ring r0 + li); its kBand2 ring-pair coefficients
// live in registers (generated through a per-thread shared-memory column).  For every map
// the CTA stages the extended spectra a_m(j) and a_m(R-1-j) of the union band as float4 in
// shared memory (one coalesced pass), then each thread sums its band with one 16-byte
// shared load and four FMAs per ring pair, predicate-free in the common case.
constexpr int kBand2 = 32;    // ring pairs per output ring held in registers
constexpr int kModes2 = 64;   // modes per CTA
constexpr int kRings2 = 8;    // representative output rings per CTA


__global__ void __launch_bounds__(kModes2 *kRings2, 2) k_contract_band(ContractArgs a, int max_union)
{
    extern __shared__ float4 sh4[];  // staging [max_union][kModes2] (aliased by the rho columns)
    float *rho_col = reinterpret_cast<float *>(sh4);
    const int tm = threadIdx.x & (kModes2 - 1);
    const int li = threadIdx.x / kModes2;
    const int m = blockIdx.x * kModes2 + tm;
    const bool mv = m < a.NH;
    const int r0 = blockIdx.y * kRings2;
    const int nr = min(kRings2, a.nrep - r0);
    const bool lv = li < nr;
    const int b0 = blockIdx.z * a.maps_per_chunk;
    const int b1 = min(a.B, b0 + a.maps_per_chunk);
    const int kid = a.per_map ? (b0 - a.map_base) : 0;
    const KernDev &kd = a.kd[kid];
    const float *taps = a.taps[kid];
    const int i = r0 + (lv ? li : 0);
    const int jl = kd.jlo[i], ps = kd.pstart[i];
    const int blen = lv ? kd.jhi[i] - jl + 1 : 0;
    const int ju0 = kd.jlo[r0];
    const int nu = kd.jhi[r0 + nr - 1] - ju0 + 1;

    // ---- coefficient generation into this thread's shared column, then registers
    for (int s = 0; s < blen; ++s) {
        const int p = ps + s;
        const int f = a.shift_fix ? kd.fl[p] : 0;
        const int S = f ? kd.S1[p] : kd.S0[p];
        const float4 *tp4 = reinterpret_cast<const float4 *>(taps + kd.toff[p]);
        float r = 0.f;
        if (mv) r = p < kd.polar_pairs ? __ldg(&a.prho[kid][(int64_t)p * a.NH + m]) : gen_rho(tp4, S, f, m, a.N);
        rho_col[s * blockDim.x + threadIdx.x] = r;
    }
    float rho[kBand2];
#pragma unroll
    for (int s = 0; s < kBand2; ++s) rho[s] = s < blen ? rho_col[s * blockDim.x + threadIdx.x] : 0.f;
    const int joff = jl - ju0;  // this ring's first input ring within the union band
    __syncthreads();

    // rows of southern rings hold (a(R-1-j), a(j)); only ring blocks whose union band crosses
    // the middle ring see them, so the swap is a block-uniform branch
    const int mid = (a.R - 1) / 2;
    const bool crosses = ju0 + nu - 1 > mid;
    const int sstar = mid - jl + 1;  // first slot of this ring's band that is a southern ring
    const size_t bufsz = (size_t)nu * kModes2;
    const int m0 = blockIdx.x * kModes2;
    if (b0 < b1) stage_band_async(sh4, map_spec4(a, b0), ju0, nu, m0, kModes2, a.R, a.NH);
    for (int b = b0; b < b1; ++b) {
        const int cur = (b - b0) & 1;
        if (b + 1 < b1)
            stage_band_async(sh4 + (cur ^ 1) * bufsz, map_spec4(a, b + 1), ju0, nu, m0,
                             kModes2, a.R, a.NH);
        else
            cp_async_commit();
        cp_async_wait1();
        __syncthreads();
        if (lv && mv) {
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 *col = sh4 + cur * bufsz + joff * kModes2 + tm;
            if (!crosses) {
#pragma unroll
                for (int s = 0; s < kBand2; ++s) {
                    if (s < blen) {
                        const float4 v = col[s * kModes2];
                        acc.x = fmaf(rho[s], v.x, acc.x);
                        acc.y = fmaf(rho[s], v.y, acc.y);
                        acc.z = fmaf(rho[s], v.z, acc.z);
                        acc.w = fmaf(rho[s], v.w, acc.w);
                    }
                }
            } else {
#pragma unroll
                for (int s = 0; s < kBand2; ++s) {
                    if (s < blen) {
                        float4 v = col[s * kModes2];
                        if (s >= sstar) v = make_float4(v.z, v.w, v.x, v.y);
                        acc.x = fmaf(rho[s], v.x, acc.x);
                        acc.y = fmaf(rho[s], v.y, acc.y);
                        acc.z = fmaf(rho[s], v.z, acc.z);
                        acc.w = fmaf(rho[s], v.w, acc.w);
                    }
                }
            }
            const int im = a.R - 1 - i;
            a.c[((int64_t)b * a.R + i) * a.NH + m] = make_float2(acc.x, acc.y);
            if (im != i) a.c[((int64_t)b * a.R + im) * a.NH + m] = make_float2(acc.z, acc.w);
        }
        __syncthreads();
    }
}

}  // namespace

int contract_ring_block() { return kRingBlock; }

int contract_band_limit() { return kBand2; }
int contract_band_rings() { return kRings2; }

cudaError_t launch_contract_band(const ContractArgs &a, int nchunks, int max_union, cudaStream_t st)
{
    const size_t smem = std::max(2 * (size_t)max_union * kModes2 * sizeof(float4),
                                 (size_t)kBand2 * kModes2 * kRings2 * sizeof(float));
    cudaError_t e = cudaFuncSetAttribute((const void *)k_contract_band,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.NH + kModes2 - 1) / kModes2, (a.nrep + kRings2 - 1) / kRings2, nchunks);
    k_contract_band<<<grid, kModes2 * kRings2, smem, st>>>(a, max_union);
    return cudaGetLastError();
}

namespace {

// Coefficients rho_m of the pairs next to the poles.  Those pairs have up to N/2 + 1 samples,
// so generating them inside the contraction would leave a few CTAs running long after the
// rest.  With x_k = pi (2k + f) / N,
//     rho_m = sum_k t_k cos(m x_k) = Re( exp(-i pi m f / N) T(m) ),  T(m) = sum_k t_k W_N^{mk},
// so for a power-of-two N one complex FFT of t_p + i t_{p+1} gives both pairs of a CTA:
// T_p(m) = (Z_m + conj Z_{N-m}) / 2 and T_{p+1}(m) = (Z_m - conj Z_{N-m}) / (2i).
template <int L>
struct PolarFft {
    const ContractArgs &a;
    float2 *buf;
    const float2 *tw;
    int kid, p0;
    __device__ void run()
    {
        constexpr int N = 1 << L;
        const KernDev &kd = a.kd[kid];
        const int np = kd.polar_pairs;
        int S[2], f[2];
        const float *tp[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int p = p0 + q;
            S[q] = -1;
            f[q] = 0;
            tp[q] = a.taps[kid];
            if (p < np) {
                f[q] = a.shift_fix ? kd.fl[p] : 0;
                S[q] = f[q] ? kd.S1[p] : kd.S0[p];
                tp[q] = a.taps[kid] + kd.toff[p];
            }
        }
        auto ld = [&](int k) {
            return make_float2(k <= S[0] ? __ldg(&tp[0][k]) : 0.f, k <= S[1] ? __ldg(&tp[1][k]) : 0.f);
        };
        fft::dif<L>(buf, tw, ld);
        const fft::Smem<L> sm{buf};
        for (int m = threadIdx.x; m < a.NH; m += blockDim.x) {
            const float2 zm = sm(fft::digitrev<L>(m)), zn = sm(fft::digitrev<L>((N - m) & (N - 1)));
            const float2 t0 = make_float2(0.5f * (zm.x + zn.x), 0.5f * (zm.y - zn.y));
            const float2 t1 = make_float2(0.5f * (zm.y + zn.y), -0.5f * (zm.x - zn.x));
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (p0 + q >= np) continue;
                const float2 t = q ? t1 : t0;
                float r = t.x;  // f = 0
                if (f[q]) {
                    const float2 e = expipi_ratio(-m, N);  // exp(-i pi m / N)
                    r = e.x * t.x - e.y * t.y;
                }
                const_cast<float *>(a.prho[kid])[(int64_t)(p0 + q) * a.NH + m] = r;
            }
        }
    }
};

__global__ void __launch_bounds__(1024) k_polar_rho_fft(ContractArgs a, const float2 *tw, int logN)
{
    extern __shared__ float2 fbuf[];
    const int kid = blockIdx.y, p0 = 2 * blockIdx.x;
    if (p0 >= a.kd[kid].polar_pairs) return;
    switch (logN) {
    case 10: PolarFft<10>{a, fbuf, tw, kid, p0}.run(); break;
    case 11: PolarFft<11>{a, fbuf, tw, kid, p0}.run(); break;
    case 12: PolarFft<12>{a, fbuf, tw, kid, p0}.run(); break;
    case 13: PolarFft<13>{a, fbuf, tw, kid, p0}.run(); break;
    default: PolarFft<14>{a, fbuf, tw, kid, p0}.run(); break;
    }
}

// The same coefficients one thread per (pair, mode), for kernel grids without the FFT form.
__global__ void __launch_bounds__(256) k_polar_rho(ContractArgs a)
{
    const int kid = blockIdx.z, p = blockIdx.y;
    const KernDev &kd = a.kd[kid];
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kd.polar_pairs || m >= a.NH) return;
    const int f = a.shift_fix ? kd.fl[p] : 0;
    const int S = f ? kd.S1[p] : kd.S0[p];
    const float4 *tp4 = reinterpret_cast<const float4 *>(a.taps[kid] + kd.toff[p]);
    const_cast<float *>(a.prho[kid])[(int64_t)p * a.NH + m] = gen_rho(tp4, S, f, m, a.N);
}

// csum[b][e] = sum_k w_k c[b K + k][e], e over the [R][NH] coefficients of a map; FP32 FMAs in
// order of k (deterministic).
struct SumWeights {
    float w[kMaxKernelsPerLaunch];
};

__global__ void __launch_bounds__(256) k_weighted_sum(const float2 *__restrict__ c, float2 *__restrict__ csum,
                                                      int K, SumWeights w, int64_t per_map, int64_t total)
{
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = idx / per_map, e = idx - b * per_map;
        float2 acc = make_float2(0.f, 0.f);
        for (int k = 0; k < K; ++k) {
            const float2 v = __ldg(&c[((int64_t)b * K + k) * per_map + e]);
            acc.x = fmaf(w.w[k], v.x, acc.x);
            acc.y = fmaf(w.w[k], v.y, acc.y);
        }
        csum[idx] = acc;
    }
}

}  // namespace

cudaError_t launch_weighted_sum(const float2 *c, float2 *csum, int64_t nmaps, int K, const double *w,
                                int64_t per_map, cudaStream_t st)
{
    if (K < 1 || K > kMaxKernelsPerLaunch) return cudaErrorInvalidValue;
    SumWeights sw;
    for (int k = 0; k < kMaxKernelsPerLaunch; ++k) sw.w[k] = k < K ? (float)w[k] : 0.f;
    const int64_t total = nmaps * per_map;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)device_sms() * 16);
    k_weighted_sum<<<blocks, 256, 0, st>>>(c, csum, K, sw, per_map, total);
    return cudaGetLastError();
}

cudaError_t launch_polar_rho(const ContractArgs &a, int nk, int max_polar_pairs, const float2 *tw, int twM,
                             cudaStream_t st)
{
    if (max_polar_pairs <= 0 || nk <= 0) return cudaSuccess;
    int logN = 0;
    while ((1 << logN) < a.N) ++logN;
    if ((1 << logN) == a.N && logN >= 10 && logN <= 14 && a.N <= twM) {
        const size_t smem = (size_t)fft::buffer_words(a.N) * sizeof(float2);
        cudaError_t e = cudaFuncSetAttribute((const void *)k_polar_rho_fft,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        dim3 grid((max_polar_pairs + 1) / 2, nk);
        k_polar_rho_fft<<<grid, a.N / 16, smem, st>>>(a, tw, logN);
        return cudaGetLastError();
    }
    dim3 grid((a.NH + 255) / 256, max_polar_pairs, nk);
    k_polar_rho<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_taps(const TapArgs &a, int npairs, cudaStream_t st)
{
    if (npairs <= 0) return cudaSuccess;
    const size_t smem = (size_t)a.kd.T * (sizeof(double) + 4 * sizeof(float));
    cudaError_t e = cudaFuncSetAttribute((const void *)k_taps,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int blocks = (npairs + 7) / 8;
    if (blocks > device_sms() * 8) blocks = device_sms() * 8;
    k_taps<<<blocks, 256, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_contract(const ContractArgs &a, int nchunks, size_t smem, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute((const void *)k_contract<kRingBlock>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.NH + kModeBlock - 1) / kModeBlock, (a.nrep + kRingBlock - 1) / kRingBlock, nchunks);
    k_contract<kRingBlock><<<grid, kModeBlock * kMapGroups, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace arkcos
