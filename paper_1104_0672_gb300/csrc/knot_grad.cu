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
#include "device_common.cuh"

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

// One warp per pair, lanes over taps: X_k = c_k sum_m cos(m x_k) Q_m, then the hat weights
// of u(x_k) deposit (1 - lam) X_k and lam X_k on knots t0, t0 + 1.  Each CTA (persistent
// over pairs) stages its deposits in shared memory and thread 0 adds them in order into the
// CTA's row of partial sums.
__global__ void __launch_bounds__(256) k_knot_proj(KnotGradArgs a, const float *Q)
{
    extern __shared__ double ksm[];
    const int T = a.kd.T;
    double *bins = ksm;             // [T]
    double *ut = ksm + T;           // [T]
    double *stage = ksm + 2 * T;    // [8 warps][32 lanes][2]
    int *stage_t = reinterpret_cast<int *>(stage + 8 * 32 * 2);
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        bins[t] = 0.0;
        ut[t] = a.kd.ut[t];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int N = a.N;
    const double invN = 1.0 / (double)N;
    // pairs are visited in rounds of (gridDim.x * nwarps); every warp of the CTA runs the same
    // number of rounds so the block-wide staging below stays in step
    const int per_round = gridDim.x * nwarps;
    const int rounds = (a.kd.npairs + per_round - 1) / per_round;
    for (int rd = 0; rd < rounds; ++rd) {
        const int p = rd * per_round + blockIdx.x * nwarps + wid;
        const bool pv = p < a.kd.npairs;
        int ntap = 0, f = 0, S = -1;
        double A = 0, B = 0;
        if (pv) {
            f = a.shift_fix ? a.kd.fl[p] : 0;
            S = f ? a.kd.S1[p] : a.kd.S0[p];
            ntap = S + 1;
            A = a.kd.A[p];
            B = a.kd.B[p];
        }
        // warp-uniform loop over tap chunks of 32; the CTA syncs once per chunk index, so
        // all warps iterate to the CTA-wide maximum chunk count
        int nchunk = (ntap + 31) >> 5;
        int maxchunk = nchunk;
        for (int o = 16; o > 0; o >>= 1) maxchunk = max(maxchunk, __shfl_xor_sync(0xffffffffu, maxchunk, o));
        __shared__ int wmax[8];
        if (lane == 0) wmax[wid] = maxchunk;
        __syncthreads();
        int cmax = 0;
        for (int w = 0; w < nwarps; ++w) cmax = max(cmax, wmax[w]);
        __syncthreads();
        for (int ch = 0; ch < cmax; ++ch) {
            const int k = ch * 32 + lane;
            double X = 0.0;
            int t0 = -1;
            double lam = 0.0;
            if (pv && k < ntap) {
                const float *q = Q + (int64_t)p * a.NH;
                // cos(m x_k), x_k = pi (2k + f) / N, by Reinsch's recurrence in m, reseeded
                // from exact values every 64 modes
                const int ang = 2 * k + f;
                float sh, chh;  // sin(x/2), cos(x/2)
                sincospif((float)ang / (float)(2 * N), &sh, &chh);
                const bool low = 2 * ang <= N;  // cos x >= 0
                const float lamr = 4.f * sh * sh, mur = 4.f * chh * chh;
                float C = 1.f, G = 0.f, acc = 0.f;
                for (int m = 0; m < a.NH; ++m) {
                    if ((m & 63) == 0) {
                        const float2 e1 = expipi_ratio(ang * m, N);
                        const float2 e2 = expipi_ratio(ang * (2 * m - 1), 2 * N);
                        C = e1.x;
                        // D_m = C_m - C_{m-1} = -2 sin((m - 1/2) x) sin(x/2);
                        // E_m = C_m + C_{m-1} = 2 cos((m - 1/2) x) cos(x/2)
                        G = low ? -2.f * e2.y * sh : 2.f * e2.x * chh;
                    } else if (low) {
                        G = fmaf(-lamr, C, G);
                        C += G;
                    } else {
                        G = fmaf(mur, C, -G);
                        C = G - C;
                    }
                    acc = fmaf(__ldg(&q[m]), C, acc);
                }
                const double mult = (f == 0 && (k == 0 || 2 * k == N)) ? 1.0 : 2.0;
                X = (double)acc * mult * invN;
                const int t = 2 * k + f;
                double u = 4.0 * (B * a.s2[N - t] + A * a.s2[t]);
                u = fmin(u, a.kd.umax);
                t0 = knot_segment(u, ut, T, a.kd.gscale);
                lam = (u - ut[t0]) / (ut[t0 + 1] - ut[t0]);
            }
            stage[(wid * 32 + lane) * 2 + 0] = (1.0 - lam) * X;
            stage[(wid * 32 + lane) * 2 + 1] = lam * X;
            stage_t[wid * 32 + lane] = t0;
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int s = 0; s < nwarps * 32; ++s) {
                    const int tt = stage_t[s];
                    if (tt >= 0) {
                        bins[tt] += stage[2 * s];
                        bins[tt + 1] += stage[2 * s + 1];
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < T; t += blockDim.x) a.partial[(int64_t)blockIdx.x * T + t] = bins[t];
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

__global__ void k_knot_reduce(const double *partial, int nrows, int T, double *out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    double s = 0.0;
    for (int r = 0; r < nrows; ++r) s += partial[(int64_t)r * T + t];
    out[t] = s;
}

}  // namespace

int knot_proj_blocks() { return 152 * 2; }

cudaError_t launch_knot_grad_q(const KnotGradArgs &a, float *Q, cudaStream_t st)
{
    dim3 grid((a.NH + kModeBlock - 1) / kModeBlock, (a.nrep + kQRing - 1) / kQRing);
    k_knot_q<<<grid, kModeBlock, 0, st>>>(a, Q);
    return cudaGetLastError();
}

cudaError_t launch_knot_grad_proj(const KnotGradArgs &a, const float *Q, cudaStream_t st)
{
    const size_t smem = (size_t)2 * a.kd.T * sizeof(double) + 8 * 32 * 2 * sizeof(double) +
                        8 * 32 * sizeof(int);
    cudaError_t e = cudaFuncSetAttribute((const void *)k_knot_proj,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_knot_proj<<<knot_proj_blocks(), 256, smem, st>>>(a, Q);
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
    k_knot_reduce<<<(T + 127) / 128, 128, 0, st>>>(partial, nrows, T, out);
    return cudaGetLastError();
}

}  // namespace arkcos
