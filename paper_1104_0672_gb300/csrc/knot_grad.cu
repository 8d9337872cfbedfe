// Gradient of J = sum_b <g_b, L r_b> with respect to the profile knots f_t.
//
// With rho_m(i,j) = sum_k c_k K_k cos(m x_k) (see contract.cu) the objective is
//     J = sum_{pairs (i,j)} sum_{m=0}^{N/2} rho_m(i,j) Q_m(i,j),
//     Q_m(i,j) = eta_m sum_b Re( w_j a_m(j,b) conj(g_m(i,b)) ),  eta = 1, 2, ..., 2, 1,
// where a and g are the (extended) ring spectra of the input maps and of the output
// gradients, so dJ/dK_k(i,j) = c_k sum_m cos(m x_k) Q_m(i,j), and K_k depends on the knots
// through the hat weights of the linear-in-u lookup.  N-S mirror pairs share their taps and
// contribute Q(i,j) + Q(R-1-i, R-1-j).  The pole rings add the derivative of their true-
// profile direct sum.  All reductions over pairs and pixels are staged per CTA and summed in
// a fixed order, so the result is bitwise reproducible.
#include "fft_engine.cuh"

namespace arkcos {

namespace {

constexpr int kQRing = 8;  // representative rings per Q CTA


// Q[p][m] for all pairs p of a block of representative rings and 128 modes (grid x: mode
// blocks, y: ring blocks).  Q is written to global memory, pairs-major.
__global__ void __launch_bounds__(kModeBlock) k_knot_q(KnotGradArgs a, float *Q)
{
    const int tid = threadIdx.x;
    const int m = blockIdx.x * kModeBlock + tid;
    if (m >= a.NH) return;
    const int r0 = blockIdx.y * kQRing;
    const int nr = min(kQRing, a.nrep - r0);
    const KernDev &kd = a.kd;
    const float eta = (m == 0 || 2 * m == a.N) ? 1.f : 2.f;
    for (int li = 0; li < nr; ++li) {
        const int i = r0 + li;
        const bool mirror = a.R - 1 - i != i;
        const bool pole = a.pole_fix && i == 0;  // ring 0 and R-1 carry no hybrid output
        const int p0 = kd.pstart[i], p1 = kd.pstart[i + 1], jl = kd.jlo[i];
        for (int p = p0; p < p1; ++p) {
            const int j = jl + (p - p0);
            float q = 0.f;
            if (!pole) {
                for (int b = 0; b < a.nmaps; ++b) {
                    const float4 *sa = a.spec4 + (int64_t)(a.map0 + b) * a.nrep * a.NH;
                    const float4 *sg = a.gspec4 + (int64_t)(a.map0 + b) * a.nrep * a.NH;
                    const float4 x = paired_coeff(sa, j, a.R, a.NH, m);   // a(j), a(R-1-j)
                    const float4 y = paired_coeff(sg, i, a.R, a.NH, m);   // g(i), g(R-1-i)
                    q = fmaf(x.x, y.x, fmaf(x.y, y.y, q));
                    if (mirror) q = fmaf(x.z, y.z, fmaf(x.w, y.w, q));
                }
            }
            Q[(int64_t)p * a.NH + m] = eta * q;
        }
    }
}

// Q for bands of at most kQBand rings: thread = (mode, representative output ring i) with
// g(i) and g(R-1-i) in registers, the union band of the input spectra staged per map in
// shared memory (double-buffered cp.async), and one accumulator per ring pair of the band.
constexpr int kQBand = 32, kQModes = 64, kQRings = 8;

__global__ void __launch_bounds__(kQModes *kQRings, 2) k_knot_q_band(KnotGradArgs a, float *Q)
{
    extern __shared__ float4 qsh[];
    const int tm = threadIdx.x & (kQModes - 1);
    const int li = threadIdx.x / kQModes;
    const int m = blockIdx.x * kQModes + tm;
    const bool mv = m < a.NH;
    const int r0 = blockIdx.y * kQRings;
    const int nr = min(kQRings, a.nrep - r0);
    const bool lv = li < nr;
    const KernDev &kd = a.kd;
    const int i = r0 + (lv ? li : 0);
    const int jl = kd.jlo[i], ps = kd.pstart[i];
    const int blen = lv ? kd.jhi[i] - jl + 1 : 0;
    const int ju0 = kd.jlo[r0];
    const int nu = kd.jhi[r0 + nr - 1] - ju0 + 1;
    const bool mirror = a.R - 1 - i != i;
    const bool pole = a.pole_fix && i == 0;  // ring 0 and R-1 carry no hybrid output
    const int mid = (a.R - 1) / 2;
    const bool crosses = ju0 + nu - 1 > mid;
    const int sstar = mid - jl + 1;
    const int joff = jl - ju0;
    const size_t bufsz = (size_t)nu * kQModes;
    const int m0 = blockIdx.x * kQModes;
    float q[kQBand];
#pragma unroll
    for (int s = 0; s < kQBand; ++s) q[s] = 0.f;
    const int b0 = a.map0, b1 = a.map0 + a.nmaps;
    if (b0 < b1) stage_band_async(qsh, a.spec4 + (int64_t)b0 * a.nrep * a.NH, ju0, nu, m0, kQModes, a.R, a.NH);
    for (int b = b0; b < b1; ++b) {
        const int cur = (b - b0) & 1;
        if (b + 1 < b1)
            stage_band_async(qsh + (cur ^ 1) * bufsz, a.spec4 + (int64_t)(b + 1) * a.nrep * a.NH, ju0, nu, m0,
                             kQModes, a.R, a.NH);
        else
            cp_async_commit();
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f);  // (g(i), g(R-1-i))
        if (lv && mv) g = __ldg(&a.gspec4[((int64_t)b * a.nrep + i) * a.NH + m]);
        if (!mirror) g.z = g.w = 0.f;
        if (pole) g = make_float4(0.f, 0.f, 0.f, 0.f);
        cp_async_wait1();
        __syncthreads();
        if (lv && mv) {
            const float4 *col = qsh + cur * bufsz + joff * kQModes + tm;
#pragma unroll
            for (int s = 0; s < kQBand; ++s) {
                if (s < blen) {
                    float4 v = col[s * kQModes];
                    if (crosses && s >= sstar) v = make_float4(v.z, v.w, v.x, v.y);
                    q[s] = fmaf(v.x, g.x, fmaf(v.y, g.y, fmaf(v.z, g.z, fmaf(v.w, g.w, q[s]))));
                }
            }
        }
        __syncthreads();
    }
    if (lv && mv) {
        const float eta = (m == 0 || 2 * m == a.N) ? 1.f : 2.f;
#pragma unroll
        for (int s = 0; s < kQBand; ++s)
            if (s < blen) Q[(int64_t)(ps + s) * a.NH + m] = eta * q[s];
    }
}

// Q for bands whose every two consecutive rings have a union band of at most kQBand rings:
// thread = (mode, group of two output rings i0 = 2g, i1 = i0 + 1 of the block) over the common
// run of kQBand input rings from jlo(i0), so each staged value feeds both rings (twice the
// arithmetic per shared-memory load of k_knot_q_band).  Rows past the block's union band stay
// zero; products outside a ring's band are accumulated but never stored.
constexpr int kQGModes = 64, kQGGroups = 4;  // 8 rings per CTA

__global__ void __launch_bounds__(kQGModes *kQGGroups, 2) k_knot_q_g2(KnotGradArgs a, float *Q, int srows)
{
    extern __shared__ float4 qgs[];  // [2 buffers][srows][kQGModes]
    const int tm = threadIdx.x & (kQGModes - 1);
    const int grp = threadIdx.x / kQGModes;
    const int m = blockIdx.x * kQGModes + tm;
    const bool mv = m < a.NH;
    const int r0 = blockIdx.y * 2 * kQGGroups;
    const int nr = min(2 * kQGGroups, a.nrep - r0);
    const KernDev &kd = a.kd;
    const int i0 = r0 + 2 * grp, i1 = i0 + 1;
    const bool v0 = 2 * grp < nr, v1 = 2 * grp + 1 < nr;  // warp-uniform (a warp is one group)
    const int jg0 = v0 ? kd.jlo[i0] : 0;
    const int ju0 = kd.jlo[r0];
    const int nu = kd.jhi[r0 + nr - 1] - ju0 + 1;
    const int joff = jg0 - ju0;
    const int mid = (a.R - 1) / 2;
    const bool crosses = ju0 + nu - 1 > mid;
    const int sstar = mid - jg0 + 1;  // first slot of the run that is a southern ring
    const size_t bufsz = (size_t)srows * kQGModes;
    const int m0 = blockIdx.x * kQGModes;
    for (size_t e = threadIdx.x; e < 2 * bufsz; e += blockDim.x) qgs[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    float q0[kQBand], q1[kQBand];
#pragma unroll
    for (int u = 0; u < kQBand; ++u) q0[u] = q1[u] = 0.f;
    // (g(i), g(R-1-i)) of a representative output ring, zero for the pole ring under the pole
    // fix (its hybrid output is replaced) and without the mirror term for the middle ring
    auto gload = [&](int b, int i, bool v) {
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
        if (v && mv) g = __ldg(&a.gspec4[((int64_t)b * a.nrep + i) * a.NH + m]);
        if (a.R - 1 - i == i) g.z = g.w = 0.f;
        if (a.pole_fix && i == 0) g = make_float4(0.f, 0.f, 0.f, 0.f);
        return g;
    };
    const int b0 = a.map0, b1 = a.map0 + a.nmaps;
    if (b0 < b1) stage_band_async(qgs, a.spec4 + (int64_t)b0 * a.nrep * a.NH, ju0, nu, m0, kQGModes, a.R, a.NH);
    for (int b = b0; b < b1; ++b) {
        const int cur = (b - b0) & 1;
        if (b + 1 < b1)
            stage_band_async(qgs + (cur ^ 1) * bufsz, a.spec4 + (int64_t)(b + 1) * a.nrep * a.NH, ju0, nu, m0,
                             kQGModes, a.R, a.NH);
        else
            cp_async_commit();
        const float4 g0 = gload(b, i0, v0), g1 = gload(b, i1, v1);
        cp_async_wait1();
        __syncthreads();
        if (v0) {
            const float4 *col = qgs + cur * bufsz + joff * kQGModes + tm;
            if (!crosses) {
#pragma unroll
                for (int u = 0; u < kQBand; ++u) {
                    const float4 v = col[u * kQGModes];
                    q0[u] = fmaf(v.x, g0.x, fmaf(v.y, g0.y, fmaf(v.z, g0.z, fmaf(v.w, g0.w, q0[u]))));
                    q1[u] = fmaf(v.x, g1.x, fmaf(v.y, g1.y, fmaf(v.z, g1.z, fmaf(v.w, g1.w, q1[u]))));
                }
            } else {
#pragma unroll
                for (int u = 0; u < kQBand; ++u) {
                    float4 v = col[u * kQGModes];
                    if (u >= sstar) v = make_float4(v.z, v.w, v.x, v.y);
                    q0[u] = fmaf(v.x, g0.x, fmaf(v.y, g0.y, fmaf(v.z, g0.z, fmaf(v.w, g0.w, q0[u]))));
                    q1[u] = fmaf(v.x, g1.x, fmaf(v.y, g1.y, fmaf(v.z, g1.z, fmaf(v.w, g1.w, q1[u]))));
                }
            }
        }
        __syncthreads();
    }
    if (v0 && mv) {
        const float eta = (m == 0 || 2 * m == a.N) ? 1.f : 2.f;
        const int ps0 = kd.pstart[i0], len0 = kd.jhi[i0] - jg0 + 1;
#pragma unroll
        for (int u = 0; u < kQBand; ++u)
            if (u < len0) Q[(int64_t)(ps0 + u) * a.NH + m] = eta * q0[u];
        if (v1) {
            const int ps1 = kd.pstart[i1], d = kd.jlo[i1] - jg0, len1 = kd.jhi[i1] - kd.jlo[i1] + 1;
#pragma unroll
            for (int u = 0; u < kQBand; ++u)
                if (u >= d && u < d + len1) Q[(int64_t)(ps1 + u - d) * a.NH + m] = eta * q1[u];
        }
    }
}

// X_k = c_k sum_m cos(m x_k) Q_m for the in-support taps of every pair, then the hat weights
// of u(x_k) deposit (1 - lam) X_k and lam X_k on knots t0, t0 + 1.
//
// Work unit = (pair, kProjTaps consecutive taps), from a table built with the kernel.  A warp
// takes one unit at a time with its lanes over the modes m = lane + 32 t (coalesced Q loads)
// and, per tap, the phasor z = exp(i m x_k) advanced by exp(i 32 x_k) each step and reseeded
// from exact values every kProjReseed steps.  The lane sums are reduced by shuffles.  The CTA's
// warps run in rounds; the round's deposits are staged in shared memory and thread 0 adds
// them in a fixed order into the CTA's shared bins, written to its row of partial sums at the
// end, so the result is reproducible.
constexpr int kProjTaps = 8, kProjReseed = 16, kProjWarps = 8;

// With Xtc (the cosine sums of pairs [pfirst, npairs) from the tensor-core product, rows of
// 128 taps) only the deposits are computed here.
__global__ void __launch_bounds__(kProjWarps * 32) k_knot_proj(KnotGradArgs a, const float *Q, const float *Xtc,
                                                               int pfirst)
{
    extern __shared__ double ksm[];
    const int T = a.kd.T;
    double *bins = ksm;                       // [T]
    double *ut = ksm + T;                     // [T]
    double *stage = ksm + 2 * T;              // [warps][kProjTaps][2]
    int *stage_t = reinterpret_cast<int *>(stage + kProjWarps * kProjTaps * 2);
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        bins[t] = 0.0;
        ut[t] = a.kd.ut[t];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int N = a.N, NH = a.NH;
    const double invN = 1.0 / (double)N;
    const int2 *units = a.shift_fix ? a.kd.unit_fix : a.kd.unit_nofix;
    const int nunits = a.shift_fix ? a.kd.nunit_fix : a.kd.nunit_nofix;
    const int per_round = gridDim.x * kProjWarps;
    const int rounds = (nunits + per_round - 1) / per_round;
    for (int rd = 0; rd < rounds; ++rd) {
        const int u = rd * per_round + blockIdx.x * kProjWarps + wid;
        double X = 0.0, lam = 0.0;
        int t0 = -1;
        if (u < nunits) {  // warp-uniform
            const int2 un = __ldg(&units[u]);
            const int p = un.x, k0 = un.y;
            const int f = a.shift_fix ? a.kd.fl[p] : 0;
            const int ntap = (f ? a.kd.S1[p] : a.kd.S0[p]) + 1;
            float mine = 0.f;
            if (Xtc) {
                if (lane < kProjTaps && k0 + lane < 128) mine = Xtc[(int64_t)(p - pfirst) * 128 + k0 + lane];
            } else {
                const float *q = Q + (int64_t)p * NH;
                float acc[kProjTaps], zr[kProjTaps], zi[kProjTaps], wr[kProjTaps], wi[kProjTaps];
#pragma unroll
                for (int j = 0; j < kProjTaps; ++j) {
                    const int ang = 2 * (k0 + j) + f;  // x = pi ang / N
                    const float2 w = expipi_ratio(32 * ang, N);
                    wr[j] = w.x;
                    wi[j] = w.y;
                    acc[j] = 0.f;
                    zr[j] = zi[j] = 0.f;
                }
                const int nsteps = (NH + 31) >> 5;
                for (int t = 0; t < nsteps; ++t) {
                    const int m = lane + 32 * t;
                    const float qm = m < NH ? __ldg(&q[m]) : 0.f;
                    if (t % kProjReseed == 0) {
#pragma unroll
                        for (int j = 0; j < kProjTaps; ++j) {
                            const float2 z = expipi_ratio((2 * (k0 + j) + f) * m, N);
                            zr[j] = z.x;
                            zi[j] = z.y;
                        }
                    }
#pragma unroll
                    for (int j = 0; j < kProjTaps; ++j) {
                        acc[j] = fmaf(qm, zr[j], acc[j]);
                        const float r = fmaf(zr[j], wr[j], -zi[j] * wi[j]);
                        zi[j] = fmaf(zr[j], wi[j], zi[j] * wr[j]);
                        zr[j] = r;
                    }
                }
#pragma unroll
                for (int j = 0; j < kProjTaps; ++j) {
                    float v = acc[j];
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == j) mine = v;
                }
            }
            const int k = k0 + lane;
            if (lane < kProjTaps && k < ntap) {
                const double mult = (f == 0 && (k == 0 || 2 * k == N)) ? 1.0 : 2.0;
                X = (double)mine * mult * invN;
                const int tt = 2 * k + f;
                double uu = 4.0 * (a.kd.B[p] * a.s2[N - tt] + a.kd.A[p] * a.s2[tt]);
                uu = fmin(uu, a.kd.umax);
                t0 = knot_segment(uu, ut, T, a.kd.gscale);
                lam = (uu - ut[t0]) / (ut[t0 + 1] - ut[t0]);
            }
        }
        if (lane < kProjTaps) {
            stage[(wid * kProjTaps + lane) * 2 + 0] = (1.0 - lam) * X;
            stage[(wid * kProjTaps + lane) * 2 + 1] = lam * X;
            stage_t[wid * kProjTaps + lane] = t0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int s = 0; s < kProjWarps * kProjTaps; ++s) {
                const int tt = stage_t[s];
                if (tt >= 0) {
                    bins[tt] += stage[2 * s];
                    bins[tt + 1] += stage[2 * s + 1];
                }
            }
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < T; t += blockDim.x) a.partial[(int64_t)blockIdx.x * T + t] = bins[t];
}

// The projection of the pairs next to the poles (up to N/2 + 1 samples each) by FFT:
//   sum_{m=0}^{N/2} Q_m cos(m x_k) = Re( sum_m Q_m e^{i pi m f / N} e^{2 pi i m k / N} ),
// one N-point inverse transform per pair (the adjoint passes from digit-reversed input), then
// the hat-weight deposits of every in-support sample.  One CTA per pair; the deposits are
// computed in parallel and added by one thread in sample order (runs of equal knots summed
// in registers), so the CTA's row of partial sums is reproducible.
template <int L>
struct ProjFft {
    const KnotGradArgs &a;
    const float *Q;
    float2 *buf;
    double *bins, *ut;
    int p, row;
    __device__ void run()
    {
        constexpr int N = 1 << L;
        const int T = a.kd.T, NH = a.NH;
        const int f = a.shift_fix ? a.kd.fl[p] : 0;
        const int ntap = (f ? a.kd.S1[p] : a.kd.S0[p]) + 1;
        const fft::Smem<L> sm{buf};
        const float *q = Q + (int64_t)p * NH;
        for (int m = threadIdx.x; m < N; m += blockDim.x) {
            float2 v = make_float2(0.f, 0.f);
            if (m < NH) {
                const float qm = __ldg(&q[m]);
                v = f ? cscalef(expipi_ratio(m, N), qm) : make_float2(qm, 0.f);
            }
            sm(fft::digitrev<L>(m), v);
        }
        __syncthreads();
        fft::adj<L>(buf, a.tw, sm);
        // this thread's samples k = tid + i blockDim: X_k and its knot segment
        constexpr int KMAX = (N / 2 + N / 16) / (N / 16);  // samples per thread (N / 16 threads)
        float xr[KMAX];
#pragma unroll
        for (int i = 0; i < KMAX; ++i) {
            const int k = threadIdx.x + i * blockDim.x;
            xr[i] = k < ntap ? sm(k).x : 0.f;
        }
        __syncthreads();
        int *t0s = reinterpret_cast<int *>(buf);
        float *w0s = reinterpret_cast<float *>(t0s + N / 2 + 1), *w1s = w0s + N / 2 + 1;
        const double invN = 1.0 / (double)N, A = a.kd.A[p], B = a.kd.B[p];
#pragma unroll
        for (int i = 0; i < KMAX; ++i) {
            const int k = threadIdx.x + i * blockDim.x;
            if (k < ntap) {
                const double mult = (f == 0 && (k == 0 || 2 * k == N)) ? 1.0 : 2.0;
                const double X = (double)xr[i] * mult * invN;
                const int t = 2 * k + f;
                double u = 4.0 * (B * a.s2[N - t] + A * a.s2[t]);
                u = fmin(u, a.kd.umax);
                const int t0 = knot_segment(u, ut, T, a.kd.gscale);
                const double lam = (u - ut[t0]) / (ut[t0 + 1] - ut[t0]);
                t0s[k] = t0;
                w0s[k] = (float)((1.0 - lam) * X);
                w1s[k] = (float)(lam * X);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int cur = -1;
            double s0 = 0.0, s1 = 0.0;
            for (int k = 0; k < ntap; ++k) {
                const int t = t0s[k];
                if (t != cur) {
                    if (cur >= 0) {
                        bins[cur] += s0;
                        bins[cur + 1] += s1;
                    }
                    cur = t;
                    s0 = s1 = 0.0;
                }
                s0 += (double)w0s[k];
                s1 += (double)w1s[k];
            }
            if (cur >= 0) {
                bins[cur] += s0;
                bins[cur + 1] += s1;
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < T; t += blockDim.x) a.partial[(int64_t)row * T + t] = bins[t];
    }
};

__global__ void __launch_bounds__(1024) k_knot_proj_fft(KnotGradArgs a, const float *Q, int logN, int row0)
{
    extern __shared__ float2 kbuf[];
    const int T = a.kd.T;
    const int N = 1 << logN;
    double *bins = reinterpret_cast<double *>(kbuf + fft::buffer_words(N));
    double *ut = bins + T;
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        bins[t] = 0.0;
        ut[t] = a.kd.ut[t];
    }
    __syncthreads();
    const int p = blockIdx.x;
    switch (logN) {
    case 10: ProjFft<10>{a, Q, kbuf, bins, ut, p, row0 + p}.run(); break;
    case 11: ProjFft<11>{a, Q, kbuf, bins, ut, p, row0 + p}.run(); break;
    case 12: ProjFft<12>{a, Q, kbuf, bins, ut, p, row0 + p}.run(); break;
    case 13: ProjFft<13>{a, Q, kbuf, bins, ut, p, row0 + p}.run(); break;
    default: ProjFft<14>{a, Q, kbuf, bins, ut, p, row0 + p}.run(); break;
    }
}

// Pole rings: d/df_t of sum_p g_p sum_q w_q K(u_pq) r_q, one CTA per (pole pixel, side, map).
__global__ void __launch_bounds__(256) k_knot_pole(KnotGradArgs a, const float *map,
                                                   const float *gout, int64_t npix, int row0)
{
    extern __shared__ double ksm[];
    const int T = a.kd.T;
    double *bins = ksm;
    double *ut = ksm + T;
    double *stage = ksm + 2 * T;
    int *stage_t = reinterpret_cast<int *>(stage + 2 * blockDim.x);
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        bins[t] = 0.0;
        ut[t] = a.kd.ut[t];
    }
    __syncthreads();
    const int p = blockIdx.x, e = blockIdx.y, b = blockIdx.z;
    const int i = e == 0 ? 0 : a.R - 1;
    const RingDev &rd = a.rd;
    const float *r = map + (int64_t)(a.map0 + b) * npix;
    const double gp = (double)gout[(int64_t)(a.map0 + b) * npix + rd.poff[i] + p];
    const int jl = a.kd.jlo[0], jh = a.kd.jhi[0];
    for (int jj = jl; jj <= jh; ++jj) {
        const int j = e == 0 ? jj : a.R - 1 - jj;
        const int nj = rd.n[j];
        for (int q0 = 0; q0 < nj; q0 += blockDim.x) {
            const int q = q0 + threadIdx.x;
            int t0 = -1;
            double lam = 0.0, X = 0.0;
            if (q < nj) {
                const double y = (double)(2 * p + rd.hs[i]) / (2.0 * rd.n[i]) -
                                 (double)(2 * q + rd.hs[j]) / (2.0 * nj);
                double sy, cy;
                sincospi(y, &sy, &cy);
                const double sd = sin(0.5 * (rd.theta[i] - rd.theta[j]));
                const double ss = sin(0.5 * (rd.theta[i] + rd.theta[j]));
                const double u = 4.0 * (sd * sd * cy * cy + ss * ss * sy * sy);
                if (u <= a.kd.umax) {
                    t0 = knot_segment(u, ut, T, a.kd.gscale);
                    lam = (u - ut[t0]) / (ut[t0 + 1] - ut[t0]);
                    X = gp * (double)rd.w[j] * (double)r[rd.poff[j] + q];
                }
            }
            stage[2 * threadIdx.x] = (1.0 - lam) * X;
            stage[2 * threadIdx.x + 1] = lam * X;
            stage_t[threadIdx.x] = t0;
            __syncthreads();
            if (threadIdx.x == 0)
                for (int s = 0; s < (int)blockDim.x; ++s)
                    if (stage_t[s] >= 0) {
                        bins[stage_t[s]] += stage[2 * s];
                        bins[stage_t[s] + 1] += stage[2 * s + 1];
                    }
            __syncthreads();
        }
    }
    const int row = row0 + (b * 2 + e) * 4 + p;
    for (int t = threadIdx.x; t < T; t += blockDim.x) a.partial[(int64_t)row * T + t] = bins[t];
}

// One CTA per knot: each thread sums a strided subset of the rows in order, then a tree over
// the threads in a fixed pairing, so the result does not depend on scheduling.
__global__ void __launch_bounds__(256) k_knot_reduce(const double *partial, int nrows, int T, double *out)
{
    __shared__ double red[256];
    const int t = blockIdx.x;
    double s = 0.0;
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) s += partial[(int64_t)r * T + t];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[t] = red[0];
}

}  // namespace

int knot_proj_blocks() { return device_sms() * 3; }
int knot_proj_taps() { return kProjTaps; }

int knot_q_band_limit() { return kQBand; }

cudaError_t launch_knot_grad_q(const KnotGradArgs &a, float *Q, int max_band, int max_union, int max_union2,
                               int srows, cudaStream_t st)
{
    const size_t smem2 = 2 * (size_t)srows * kQGModes * sizeof(float4);
    if (max_union2 <= kQBand && smem2 <= 100 * 1024) {
        cudaError_t e = cudaFuncSetAttribute((const void *)k_knot_q_g2,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
        if (e != cudaSuccess) return e;
        dim3 grid((a.NH + kQGModes - 1) / kQGModes, (a.nrep + 2 * kQGGroups - 1) / (2 * kQGGroups));
        k_knot_q_g2<<<grid, kQGModes * kQGGroups, smem2, st>>>(a, Q, srows);
        return cudaGetLastError();
    }
    const size_t smem = 2 * (size_t)max_union * kQModes * sizeof(float4);
    if (max_band <= kQBand && smem <= 200 * 1024) {
        cudaError_t e = cudaFuncSetAttribute((const void *)k_knot_q_band,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        dim3 grid((a.NH + kQModes - 1) / kQModes, (a.nrep + kQRings - 1) / kQRings);
        k_knot_q_band<<<grid, kQModes * kQRings, smem, st>>>(a, Q);
        return cudaGetLastError();
    }
    dim3 grid((a.NH + kModeBlock - 1) / kModeBlock, (a.nrep + kQRing - 1) / kQRing);
    k_knot_q<<<grid, kModeBlock, 0, st>>>(a, Q);
    return cudaGetLastError();
}

cudaError_t launch_knot_grad_proj(const KnotGradArgs &a, const float *Q, const float *X, int pfirst,
                                  cudaStream_t st)
{
    const size_t smem = (size_t)2 * a.kd.T * sizeof(double) + kProjWarps * kProjTaps * 2 * sizeof(double) +
                        kProjWarps * kProjTaps * sizeof(int);
    cudaError_t e = cudaFuncSetAttribute((const void *)k_knot_proj,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_knot_proj<<<knot_proj_blocks(), kProjWarps * 32, smem, st>>>(a, Q, X, pfirst);
    return cudaGetLastError();
}

// Pairs [0, npairs) by FFT (the caller checks that N is a power of two in [2^10, 2^14] and
// within the grid's twiddle table); their rows of partial sums start at row0.
cudaError_t launch_knot_grad_proj_fft(const KnotGradArgs &a, const float *Q, int npairs, int row0, cudaStream_t st)
{
    if (npairs <= 0) return cudaSuccess;
    int logN = 0;
    while ((1 << logN) < a.N) ++logN;
    const size_t smem = (size_t)fft::buffer_words(a.N) * sizeof(float2) + 2 * (size_t)a.kd.T * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute((const void *)k_knot_proj_fft,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_knot_proj_fft<<<npairs, a.N / 16, smem, st>>>(a, Q, logN, row0);
    return cudaGetLastError();
}

cudaError_t launch_knot_grad_pole(const KnotGradArgs &a, const float *map, const float *gout,
                                  int64_t npix, int row0, cudaStream_t st)
{
    const size_t smem = (size_t)2 * a.kd.T * sizeof(double) + 256 * 2 * sizeof(double) +
                        256 * sizeof(int);
    cudaError_t e = cudaFuncSetAttribute((const void *)k_knot_pole,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(4, 2, a.nmaps);
    k_knot_pole<<<grid, 256, smem, st>>>(a, map, gout, npix, row0);
    return cudaGetLastError();
}

cudaError_t launch_knot_reduce(const double *partial, int nrows, int T, double *out, cudaStream_t st)
{
    k_knot_reduce<<<T, 256, 0, st>>>(partial, nrows, T, out);
    return cudaGetLastError();
}

}  // namespace arkcos
